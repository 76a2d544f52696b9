/*
 * bsgdtv.h -- C ABI of the GB300 (sm_103a) BSGD-TV library.
 *
 * BSGD-TV (Gao & Blumensath, arXiv 1812.01307) reconstructs an image x from
 * projections y ~ A x by repeating one epoch of Algorithm 1:
 *   block products  z^j_{I_i} = A_{I_i}^{J_j} x_{J_j}  and
 *                   g^i_{J_j} = 2 (A_{I_i}^{J_j})^T r_{I_i}   (r from the previous epoch)
 *   residual        r = y - sum_j z^j
 *   gradient        g = sum_i g^i
 *   step            x = x + mu g
 *   TV prox         x = argmin_t ||t - x||^2 + 2 mu lambda TV(t), solved by Beck &
 *                   Teboulle's fast gradient projection (FGP) with tau = mu*lambda.
 * A is divided into M row blocks I_i and N column blocks J_j (Sec. 2.1).
 *
 * Conventions shared by every entry point
 *   - Return value: BSGDTV_OK (0) or a negative BSGDTV_ERR_* code.  Nothing
 *     throws across this boundary.  bsgdtv_last_error() gives a message for
 *     the calling thread's most recent failure.
 *   - Host arrays passed in are copied; the caller keeps ownership.  A handle
 *     owns all the device memory it allocates and frees it in bsgdtv_destroy.
 *   - `*_on_device` flags say whether a pointer is device memory (1) or host
 *     memory (0).  Device pointers must be on the handle's device.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *     call enqueues its work on the handle's stream; calls that return data to
 *     the host (get_x to host, objective, estimate_umax, ...) synchronise it.
 *   - The image is img_h x img_w, row-major (pixel (s,t) is column s*img_w+t
 *     of A).  TV is isotropic with forward differences and a zero-difference
 *     (Neumann) border, the discretisation FGP is defined on.
 *   - Floating point: A values, x, y, r are FP32 with FP32 accumulation on the
 *     hot path; u_max and the objective are computed in FP64.
 *   - Threads: calls on one handle (bsgdtv_t, bsgdtv_batch_t) must not
 *     overlap; different handles may be used from different threads.  The
 *     server (bsgdtv_server_t) accepts calls from any thread at any time.
 */
#ifndef BSGDTV_H
#define BSGDTV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsgdtv_ctx *bsgdtv_t;

enum {
    BSGDTV_OK = 0,
    BSGDTV_ERR_INVALID_ARG = -1, /* bad size, pointer, bound or flag */
    BSGDTV_ERR_OOM = -2,         /* device or host allocation failed */
    BSGDTV_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    BSGDTV_ERR_STATE = -4,       /* call out of order (e.g. run before set_data) */
    BSGDTV_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    BSGDTV_ERR_NONFINITE = -6,   /* NaN/Inf in an input */
    BSGDTV_ERR_UNSUPPORTED = -7, /* valid request the library does not handle */
    BSGDTV_ERR_CANCELLED = -8    /* a server request was cancelled */
};

/* How the device stores A's weights and tile-local column indices.  F32_I32
 * keeps FP32 weights and 32-bit indices (8 bytes per nonzero); F32_I16 is the
 * same operator with 16-bit indices (6 bytes, exact); F16_I16 and BF16_I16
 * round the weights to IEEE binary16 / bfloat16 (round to nearest even, 4
 * bytes per nonzero) and compute in FP32 from the rounded values. */
enum {
    BSGDTV_FMT_F32_I32 = 0,
    BSGDTV_FMT_F32_I16 = 1,
    BSGDTV_FMT_F16_I16 = 2,
    BSGDTV_FMT_BF16_I16 = 3
};

/* Creates a handle from a host CSR matrix A (rows = rays, cols = pixels; the
 * system y = A x of Eq. 1) split into the M x N blocks A_{I_i}^{J_j} of
 * Sec. 2.1.
 *   rows, cols          size of A; cols must equal img_h*img_w.
 *   row_ptr [rows+1]    int64 offsets, row_ptr[0] = 0, non-decreasing.
 *   col_idx [nnz]       int32 column indices in [0, cols), ascending in a row.
 *   vals    [nnz]       float64 weights (stored on the device as FP32).
 *   M, N                number of row / column blocks (Sec. 2.1).
 *   row_bounds [M+1]    optional explicit I_i bounds (NULL: numpy.array_split of
 *                       rows/row_unit units into M groups, times row_unit).
 *   col_bounds [N+1]    optional explicit J_j bounds (NULL: the same with
 *                       cols/col_unit and N).  Every J_j bound must be a multiple
 *                       of img_w: column blocks are bands of whole image rows.
 *   row_unit, col_unit  grouping units for the default bounds (e.g. n_bins and
 *                       img_w so that I_i are whole angles, J_j whole rows).
 *   stream              cudaStream_t for all of this handle's work.
 * Validates the CSR (sorted, in range, finite) and fails with
 * BSGDTV_ERR_INVALID_ARG / BSGDTV_ERR_NONFINITE otherwise. */
int bsgdtv_create_csr(bsgdtv_t *out, int64_t rows, int64_t cols, int img_h, int img_w,
                      const int64_t *row_ptr, const int32_t *col_idx, const double *vals,
                      int M, int N, int64_t row_unit, int64_t col_unit,
                      const int64_t *row_bounds, const int64_t *col_bounds, void *stream);

/* bsgdtv_create_csr with a stored format (BSGDTV_FMT_*); create_csr uses
 * BSGDTV_FMT_F32_I32.  u_max, the objective and every product of the handle
 * use the stored (rounded) weights. */
int bsgdtv_create_csr_ex(bsgdtv_t *out, int64_t rows, int64_t cols, int img_h, int img_w,
                         const int64_t *row_ptr, const int32_t *col_idx, const double *vals,
                         int M, int N, int64_t row_unit, int64_t col_unit,
                         const int64_t *row_bounds, const int64_t *col_bounds, int format,
                         void *stream);

/* bsgdtv_create_csr_ex for the 2-D parallel-beam geometry of an n x n image
 * (pixel size 1, centred at the origin), n_angles angles k*pi/n_angles and
 * n_bins unit detector bins centred on the origin: A (rows k*n_bins + d,
 * columns s*n + t) holds the exact intersection lengths of ray and pixel,
 * generated on the device by the matrix-free projector of
 * bsgdtv_batch_create_parallel_beam (each weight within about 1e-7 of its
 * FP64 value; half-open pixels, |sin|, |cos| < 1e-15 taken as 0) and stored in
 * `format`.  Row blocks are M groups of whole angles, column blocks N bands
 * of whole image rows (the array_split rule).  Needs host memory for the
 * CSR (12 bytes per nonzero) while the handle is built. */
int bsgdtv_create_parallel_beam(bsgdtv_t *out, int n, int n_angles, int n_bins, int M, int N,
                                int format, void *stream);

/* Releases every resource of the handle (API housekeeping: no passage of
 * the paper).  NULL is ignored. */
void bsgdtv_destroy(bsgdtv_t h);

/* Copies the partition bounds I_i [M+1] and J_j [N+1] of Sec. 2.1 (host
 * arrays, either may be NULL). */
int bsgdtv_get_partition(bsgdtv_t h, int64_t *row_bounds, int64_t *col_bounds);

/* Sets the projections y [rows] (FP32; Eq. 1), the TV weight lambda >= 0
 * (Eq. 1, Algorithm 1's prox weight 2 mu lambda) and the step mu.  mu <= 0 selects mu = 0.9/(2 u_max) (Theorem 1 requires mu < 1/(2 u_max)),
 * estimating u_max first if no estimate exists.  Resets the iteration:
 * x^0 = 0, r^{-1} = y - A x^0 = y, epoch counter 0.  Rejects NaN/Inf in y
 * (BSGDTV_ERR_NONFINITE); once y is being copied, a failure leaves the handle
 * without data (bsgdtv_run returns BSGDTV_ERR_STATE until a set_data
 * succeeds).  A host y may be reused as soon as the call returns, pinned or
 * not (the call waits for the handle's earlier work and the copy). */
int bsgdtv_set_data(bsgdtv_t h, const float *y, int y_on_device, double lambda, double mu);

/* Largest eigenvalue u_max of A^T A (Theorem 1: the epoch recurrence
 * converges for mu < 1/(2 u_max)) by power iteration in FP64 on the device
 * (A as stored, i.e. FP32 weights widened to FP64), from the all-ones vector,
 * stopping when the Rayleigh quotient changes by <= rel_tol relatively or after
 * max_iters iterations.  Writes u_max and the iteration count (may be NULL). */
int bsgdtv_estimate_umax(bsgdtv_t h, int max_iters, double rel_tol, double *u_max, int *iters);

/* Current step mu (after set_data) and the stored u_max estimate (0 if none). */
int bsgdtv_get_params(bsgdtv_t h, double *mu, double *lambda, double *u_max);

/* Runs `epochs` epochs of Algorithm 1 (Sec. 2.1: block products, residual
 * and gradient sums, step, TV prox; the gradient uses the previous epoch's
 * residual, Eq. 3) with `fgp_iters` FGP iterations for the TV prox (lambda =
 * 0 or fgp_iters = 0 makes the prox the identity).  Asynchronous
 * on the handle's stream; resumes from the current state. */
int bsgdtv_run(bsgdtv_t h, int epochs, int fgp_iters);

/* The stochastic variant of Sec. 3: `iters` iterations in which only the
 * drawn row blocks (row_sel [iters][M], nonzero = drawn) and column blocks
 * (col_sel [iters][N]) take part; the draws are the caller's (host arrays).
 * Iteration k: the pairs (i, j) with both drawn form their block products
 * from the current x and r; r on the drawn row blocks becomes
 * y - sum_j z^j with z^j of undrawn j the last one computed (0 after
 * set_data, consistent with x^0 = 0); x on the drawn column blocks gains
 * mu * sum over drawn i of g-hat^i; other parts of r and x are unchanged; the
 * TV prox then acts on the whole image.  With every block drawn it is
 * bsgdtv_run.  Every iteration must draw at least one row and one column
 * block (else BSGDTV_ERR_INVALID_ARG).  Counts iterations in the epoch
 * counter; synchronises before returning (the host arrays may be freed). */
int bsgdtv_run_subsets(bsgdtv_t h, int iters, int fgp_iters, const uint8_t *row_sel,
                       const uint8_t *col_sel);

/* bsgdtv_run_subsets with its device time: *device_ms receives the CUDA-event
 * time on the handle's stream from the moment the work-item lists are on the
 * device to the end of the last iteration's kernels; *prep_ms (may be NULL)
 * the host time spent validating the draws and building and uploading the
 * lists.  Same iterates as bsgdtv_run_subsets; synchronises. */
int bsgdtv_run_subsets_timed(bsgdtv_t h, int iters, int fgp_iters, const uint8_t *row_sel,
                             const uint8_t *col_sel, double *device_ms, double *prep_ms);

/* bsgdtv_run that also times, with CUDA events recorded on the handle's
 * stream inside the epoch graphs, every launch of the fused product kernel
 * (the block products) and every whole epoch.  Synchronises.  products_ms / epoch_ms
 * (may be NULL) receive the sums over the `epochs` epochs. */
int bsgdtv_run_timed(bsgdtv_t h, int epochs, int fgp_iters, double *products_ms,
                     double *epoch_ms);

/* Copies the current iterate x^k of Algorithm 1, [cols] FP32, row-major
 * image, into out (n floats: BSGDTV_ERR_INVALID_ARG if n < cols).  To the
 * host: synchronises the stream. */
int bsgdtv_get_x(bsgdtv_t h, float *out, int out_on_device, int64_t n);

/* One reconstruction in one call: bsgdtv_set_data(y, lambda, mu), then
 * bsgdtv_run(epochs, fgp_iters) (Algorithm 1, Sec. 2.1), then bsgdtv_get_x
 * into x_out (n_x floats, at least cols), queued on the handle's stream and
 * synchronised once at the end instead of after the copy of y and again after
 * the copy of x.  Same iterates as the three calls.  The check of y for
 * NaN/Inf is read back with x: non-finite y gives BSGDTV_ERR_NONFINITE after
 * the epochs have run (x_out then holds no meaningful result) and leaves the
 * handle without data, as a failed set_data does.  A host y and x_out may be
 * reused as soon as the call returns. */
int bsgdtv_reconstruct(bsgdtv_t h, const float *y, int y_on_device, double lambda, double mu,
                       int epochs, int fgp_iters, float *x_out, int x_on_device, int64_t n_x);

/* Checkpoint: x^k [cols], r^{k-1} [rows] (the residual the next epoch's
 * gradient uses: Eq. 3 makes it part of the state) and k.  set_state restores them (requires set_data first). */
int bsgdtv_get_state(bsgdtv_t h, float *x, float *r, int64_t *epoch, int on_device);
int bsgdtv_set_state(bsgdtv_t h, const float *x, const float *r, int64_t epoch, int on_device);

/* FP64 monitoring of the current x: data term ||y - A x||^2 and TV(x)
 * (Eq. 1, TV of Eq. 2 read as isotropic forward differences with a Neumann
 * border; the function Algorithm 1 with its TV prox as printed minimises is
 * data + lambda*TV).
 * Synchronises. */
int bsgdtv_objective(bsgdtv_t h, double *data_term, double *tv);

/* Runs epochs as bsgdtv_run does, in steps of check_every (>= 1) epochs,
 * evaluating the FP64 objective F = ||y - A x||^2 + lambda TV(x)
 * (bsgdtv_objective) before the first step and after each one, and stops
 * after the step where |F_before - F_after| <= rel_tol * F_before, or once
 * max_epochs have run (the last step may be shorter).  Writes the epochs run
 * and the last F (either may be NULL).  The iterates are those of
 * bsgdtv_run for the same number of epochs, bit for bit.  Synchronises at
 * every check.  The stopping rule is a deployment choice; the paper runs
 * fixed epoch counts. */
int bsgdtv_run_until(bsgdtv_t h, int max_epochs, int fgp_iters, int check_every, double rel_tol,
                     int *epochs_run, double *objective);

/* Test hook: the block products z^j_{I_i} and g-hat^i_{J_j} of Algorithm 1
 * (Sec. 2.1) for given x [cols] and r [rows]
 * (device pointers), computed by the same fused kernel the epoch uses.
 *   z_blocks [N*rows]:  z_blocks[j*rows + k] = (A_{I_i}^{J_j} x_{J_j})_k for row
 *                       k of block I_i (i.e. z^j stacked over i).
 *   g_blocks [M*cols]:  g_blocks[i*cols + c] = (2 (A_{I_i}^{J_j})^T r_{I_i})_c
 *                       for column c of block J_j.
 * Does not touch the iteration state. */
int bsgdtv_block_products(bsgdtv_t h, const float *x, const float *r, float *z_blocks,
                          float *g_blocks);

/* Sizes of the stored operator: nnz of A, number of row segments in the tiled
 * layout, work items per product pass, and the bytes one product pass must
 * move at minimum (the format's bytes per nonzero + x, r, z, g once). */
int bsgdtv_get_info(bsgdtv_t h, int64_t *nnz, int64_t *segments, int64_t *work_items,
                    int64_t *min_bytes_per_pass);

/* The TV prox alone: x = FGP(b, tau, iters) for one img_h x img_w image (device
 * pointers b, x; may not alias).  Beck-Teboulle FGP, cold start, isotropic TV,
 * P_C = identity; tau <= 0 or iters == 0 copies b; iters < 0 (or a
 * non-finite tau) is BSGDTV_ERR_INVALID_ARG.  Allocates its scratch (the
 * dual fields) from the device heap for the duration of the call and
 * synchronises `stream` before returning. */
int bsgdtv_tv_prox(const float *b, float *x, int img_h, int img_w, double tau, int iters,
                   void *stream);

/* bsgdtv_tv_prox for callers that cannot allocate device memory at call
 * time (the paper has no counterpart; this is a deployment variant).  Such
 * callers include processes whose device budget is fully claimed by their own
 * pool allocator, latency-critical loops that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree, and host runtimes that forbid
 * plugins from allocating.  Same arguments, same result as bsgdtv_tv_prox;
 * it calls no cudaMalloc, cudaFree or other allocating routine.  Its scratch
 * (two sets of FGP dual fields and the momentum table) is one file-scope
 * device array of about 8 MiB that every GPU which loads the library keeps until the process
 * exits.  Limits: img_h*img_w <= 262144 (e.g. 512 x 512) and iters <= 4096;
 * larger requests fail with BSGDTV_ERR_INVALID_ARG.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls
 * in the process share the one array and it keeps the last call's contents
 * (nothing in it needs to start at zero): calls that overlap on the GPU, e.g.
 * on two streams or from two threads, race.  Synchronises `stream`. */
int bsgdtv_tv_prox_static(const float *b, float *x, int img_h, int img_w, double tau, int iters,
                          void *stream);

/* Host only (no GPU needed): how the TV prox (Beck-Teboulle FGP, the prox of
 * Algorithm 1's last step) tiles one image dimension of len pixels into
 * regions of 64 pixels that overlap by `halo` (iterations per launch + 1):
 * the region count, and for the first max_regions regions k their first
 * pixel first[k] and their interior [lo[k], hi[k]) in region coordinates
 * (first, lo, hi may be NULL).  The regions at the image's edges keep no halo
 * on the outer side.  This is the placement the prox kernel computes. */
int bsgdtv_fgp_tiling(int len, int halo, int max_regions, int *n_regions, int *first, int *lo,
                      int *hi);

/* Host only (no GPU needed): the partition bounds bsgdtv_create_csr uses when
 * row_bounds / col_bounds are NULL, written to row_bounds [M+1] and
 * col_bounds [N+1]. */
int bsgdtv_partition_bounds(int64_t rows, int64_t cols, int M, int N, int64_t row_unit,
                            int64_t col_unit, int64_t *row_bounds, int64_t *col_bounds);

/* Host only (no GPU needed): validates a CSR exactly as bsgdtv_create_csr
 * does, builds the tiled device layout in host memory and checks that decoding
 * it gives back A (columns exact, values equal to the FP32-rounded input).
 * stats [6] (may be NULL) receives {nnz, segments, slabs, work items, row
 * groups, pixel tiles}.  Returns BSGDTV_ERR_INVALID_ARG / _NONFINITE for a bad
 * CSR and BSGDTV_ERR_STATE if the layout does not reproduce A (with the
 * weights rounded to `format`). */
int bsgdtv_layout_check(int64_t rows, int64_t cols, int img_h, int img_w, const int64_t *row_ptr,
                        const int32_t *col_idx, const double *vals, int M, int N,
                        int64_t row_unit, int64_t col_unit, const int64_t *row_bounds,
                        const int64_t *col_bounds, int format, int target_items,
                        int64_t *stats);

/* Host only: the weight as a handle of the given format stores it, widened to
 * FP32 (round to nearest even for the 16-bit formats). */
float bsgdtv_stored_weight(double v, int format);

/* Measured FP32 CUDA-core throughput of the current device, in TFLOP/s (2
 * flops per FMA): independent FMA chains at full occupancy, timed with CUDA
 * events on a private stream, best of three runs after a warm-up, once with
 * scalar FMAs (*tflops_scalar) and once with packed two-lane FMAs
 * (*tflops_packed; either may be NULL).  The denominator of the ALU
 * rooflines of the batched and matrix-free product passes.  Allocates and
 * frees a small output buffer; synchronises. */
int bsgdtv_fp32_fma_peak(double *tflops_scalar, double *tflops_packed);

/* Number of kernels this library has launched in the calling process
 * (graph replays count every kernel node). */
int64_t bsgdtv_launch_count(void);

/* Message for the calling thread's most recent failure ("" if none). */
const char *bsgdtv_last_error(void);

/* Static description of an error code. */
const char *bsgdtv_strerror(int code);

/* ------------------------------------------------------------ batched slices
 * B independent reconstructions (e.g. the slices of a parallel-beam volume)
 * that share one matrix A: slice b has projections y_b, TV weight lambda_b,
 * iterate x_b and residual r_b, and every slice uses the same step mu.  Each
 * slice follows Algorithm 1 exactly as a single-slice handle does (x^0 = 0,
 * r^{-1} = y_b, stale residual in the gradient, FGP prox with
 * tau_b = mu*lambda_b); the block partition of Sec. 2.1 changes only how the
 * work is divided, not the iterates, so a batch has no M, N.  Both products of
 * an epoch come from one pass over A each (in CSR for A x, in CSC for A^T r)
 * that applies every nonzero to all B slices, with FP32 accumulation in a
 * fixed order (deterministic).  Device memory: A twice (12 bytes per nonzero
 * each) plus about 4 (rows + cols) Bp + 7 cols B floats, Bp = B rounded up to
 * 32, 64 or a multiple of 128. */
typedef struct bsgdtv_batch_ctx *bsgdtv_batch_t;

/* A, stored once on the device for batches of any size: a reference-counted
 * operator.  bsgdtv_operator_create_csr validates and uploads a host CSR A
 * (arguments as for bsgdtv_batch_create_csr_ex, weights in `format`);
 * bsgdtv_batch_create_from_operator builds a batch that reads it (and holds a
 * reference, so the creator may call bsgdtv_operator_destroy at any time; the
 * device arrays go when the last batch using them is destroyed).  A batch from
 * an operator allocates only its vectors (bsgdtv_batch_device_bytes with
 * nnz = 0).  Batches on one operator may run concurrently on different
 * streams: they only read it. */
typedef struct bsgdtv_operator_ctx *bsgdtv_operator_t;

int bsgdtv_operator_create_csr(bsgdtv_operator_t *out, int64_t rows, int64_t cols, int img_h,
                               int img_w, const int64_t *row_ptr, const int32_t *col_idx,
                               const double *vals, int format, void *stream);
void bsgdtv_operator_destroy(bsgdtv_operator_t op);
int bsgdtv_batch_create_from_operator(bsgdtv_batch_t *out, bsgdtv_operator_t op, int slices,
                                      void *stream);

/* Creates a batch of `slices` (1 .. 4096) slices from a host CSR matrix A; the
 * arguments rows .. vals and `stream` mean what they mean for
 * bsgdtv_create_csr (A stored as FP32 weights, 32-bit indices).  Fails with
 * BSGDTV_ERR_INVALID_ARG / BSGDTV_ERR_NONFINITE on a malformed CSR. */
int bsgdtv_batch_create_csr(bsgdtv_batch_t *out, int64_t rows, int64_t cols, int img_h, int img_w,
                            const int64_t *row_ptr, const int32_t *col_idx, const double *vals,
                            int slices, void *stream);

/* bsgdtv_batch_create_csr with a weight format: BSGDTV_FMT_F32_I32 (FP32
 * weights, 8 bytes per nonzero and pass), BSGDTV_FMT_F16_I16 or
 * BSGDTV_FMT_BF16_I16 (weights rounded to nearest even binary16 / bfloat16,
 * 6 bytes per nonzero and pass, FP32 arithmetic).  A batch always keeps
 * 32-bit element offsets, so the index width in the format's name does not
 * apply; BSGDTV_FMT_F32_I16 is BSGDTV_ERR_UNSUPPORTED here. */
int bsgdtv_batch_create_csr_ex(bsgdtv_batch_t *out, int64_t rows, int64_t cols, int img_h,
                               int img_w, const int64_t *row_ptr, const int32_t *col_idx,
                               const double *vals, int slices, int format, void *stream);

/* Host only: the device bytes a batch of these sizes allocates (A twice,
 * the interleaved and planar vectors, FGP fields), within a few KiB; -1 on
 * bad sizes; nnz = 0 for a matrix-free batch.  Used for admission by free
 * memory. */
int64_t bsgdtv_batch_device_bytes(int64_t rows, int64_t cols, int64_t nnz, int slices, int format);

/* A matrix-free batch for the 2-D parallel-beam geometry of an n x n image
 * (pixel size 1, centred), n_angles angles k*pi/n_angles and n_bins unit
 * detector bins centred on the origin: the weights of A (exact intersection
 * lengths of ray and pixel, the convention of the stored-matrix generator:
 * half-open pixels, |sin|, |cos| < 1e-15 taken as 0) are computed on the fly
 * in both passes, so A takes no device memory.  Rows are k*n_bins + d,
 * columns s*n + t.  Each weight is formed in compensated FP32 and agrees with
 * the FP64 intersection length to about 1e-7; the row and column passes use
 * bit-identical weights.  Everything else is as for bsgdtv_batch_create_csr. */
int bsgdtv_batch_create_parallel_beam(bsgdtv_batch_t *out, int n, int n_angles, int n_bins,
                                      int slices, void *stream);

/* Test hook: the weights the matrix-free row pass uses for the listed rays
 * (host rays [n_rays], row indices), written per ray i to cols / vals
 * [i*capacity ...] (host, n_rays*capacity entries) in the pass's order, with
 * counts[i] entries (at most capacity kept).  Synchronous. */
int bsgdtv_mf_ray_weights(int n, int n_angles, int n_bins, const int64_t *rays, int n_rays,
                          int capacity, int32_t *cols, float *vals, int *counts);

/* Largest eigenvalue u_max of A^T A for a batch's A (stored or matrix free)
 * by power iteration from the all-ones vector on the batch's own passes (FP32
 * products, FP64 norms and Rayleigh quotients), stopping at relative change
 * <= rel_tol or max_iters.  Uses the batch's vectors as scratch: every slice
 * must be set again (bsgdtv_batch_set_data) afterwards. */
int bsgdtv_batch_estimate_umax(bsgdtv_batch_t h, int max_iters, double rel_tol, double *u_max,
                               int *iters);

/* Releases every resource of the batch.  NULL is ignored. */
void bsgdtv_batch_destroy(bsgdtv_batch_t h);

/* Sets every slice's projections y [slices][rows] (slice-major FP32), the
 * weights lambdas [slices] (host, each finite and >= 0) and the step mu > 0
 * (finite; Theorem 1 asks mu < 1/(2 u_max), with u_max from
 * bsgdtv_estimate_umax of a single-slice handle on the same A).  Resets every
 * slice: x^0 = 0, r^{-1} = y_b.  Rejects NaN/Inf in y (BSGDTV_ERR_NONFINITE);
 * once y is being copied a failure leaves the batch without data.  Returns
 * after y has been read (a host y may be reused at once, pinned or not). */
int bsgdtv_batch_set_data(bsgdtv_batch_t h, const float *y, int y_on_device,
                          const double *lambdas, double mu);

/* Runs `epochs` epochs of Algorithm 1 on every slice, with `fgp_iters` FGP
 * iterations for each prox (a slice with lambda_b = 0, or fgp_iters = 0, has
 * the identity prox).  Asynchronous on the batch's stream; resumes from the
 * current state.  BSGDTV_ERR_STATE before set_data. */
int bsgdtv_batch_run(bsgdtv_batch_t h, int epochs, int fgp_iters);

/* bsgdtv_batch_run that also times, with CUDA events recorded on the stream
 * inside the epoch graphs, the two product passes of every epoch and every
 * whole epoch.  Synchronises.  products_ms / epoch_ms (may be NULL) receive
 * the sums over the `epochs` epochs. */
int bsgdtv_batch_run_timed(bsgdtv_batch_t h, int epochs, int fgp_iters, double *products_ms,
                           double *epoch_ms);

/* Copies every slice's x into x [slices][cols] (slice-major FP32).  To the
 * host: synchronises the stream. */
int bsgdtv_batch_get_x(bsgdtv_batch_t h, float *x, int out_on_device);

/* Restarts slice b alone (a slot of a continuously batched server): y_b
 * [rows] (FP32, host or device) and lambda >= 0 replace the slice's data and
 * the slice resets to x^0 = 0, r^{-1} = y_b; the step mu stays the one of
 * set_data.  y = NULL empties the slot (y = x = r = 0, lambda = 0).  The other
 * slices are untouched, and since every slice's arithmetic is independent of
 * the others, a slice's iterates do not depend on what the other slots hold.
 * Stream-ordered with run; BSGDTV_ERR_STATE before set_data.  A host y is
 * checked for NaN/Inf (BSGDTV_ERR_NONFINITE leaves the slot as it was) and
 * may be reused when the call returns. */
int bsgdtv_batch_set_slice(bsgdtv_batch_t h, int b, const float *y, int y_on_device, double lambda);

/* Forward projection y_b = A x_b of every slice with the batch's A (stored
 * or matrix free): x [slices][cols] and y [slices][rows], both device FP32,
 * slice-major.  Uses the batch's vectors as scratch: every slice must be set
 * again (bsgdtv_batch_set_data) afterwards.  Synchronises. */
int bsgdtv_batch_project(bsgdtv_batch_t h, const float *x, float *y);

/* Autotuner: times epochs_per_trial epochs of this batch (on its current
 * data, state restored after every trial) for each candidate launch shape
 * and keeps the fastest.  First the lanes per nonzero of each product pass
 * (the batch's own count, half and a quarter of it: slices per warp step,
 * see bsgdtv_batch_set_pass_lanes; these change the order of FP32 sums, so
 * results may move within FP32 rounding), then the FGP iterations per
 * launch (3, 4, 5, 6, 8: fewer iterations per launch mean a smaller halo per
 * 64 x 64 region but more launches and field traffic) times the slices per
 * FGP launch group (half, once and twice the count whose dual fields fill
 * 48 MB of L2, and all slices: small groups keep the fields in L2, large
 * ones fill more SMs per launch; these give bit-identical iterates).  Writes
 * the FGP choices and the time per epoch (each may be NULL;
 * bsgdtv_batch_get_tuning has all choices).  Synchronises; needs set_data. */
int bsgdtv_batch_autotune(bsgdtv_batch_t h, int fgp_iters, int epochs_per_trial, int *fgp_chunk,
                          int *fgp_group, double *epoch_ms);

/* Applies a known tuning without timing (e.g. one bsgdtv_batch_autotune found
 * earlier): FGP iterations per launch 1..8 (0: the default) and slices per
 * FGP launch group (0: sized by the 48 MB L2 budget).  Results do not depend
 * on it.  Synchronises the stream when the tuning changes. */
int bsgdtv_batch_set_tuning(bsgdtv_batch_t h, int fgp_chunk, int fgp_group);

/* The tuning in force: FGP iterations per launch, slices per FGP launch
 * group, and the lanes per nonzero of the row and column passes (any output
 * may be NULL). */
int bsgdtv_batch_get_tuning(bsgdtv_batch_t h, int *fgp_chunk, int *fgp_group, int *lanes_row,
                            int *lanes_col);

/* Lanes per nonzero of the row and column passes: each lane carries 4
 * slices, so with L lanes a warp applies 32 / L nonzeros per step to 4 L
 * slices and takes the padded slices in Bp / (4 L) chunks.  0 restores the
 * batch's own count (the smallest with 4 L >= slices, at most 32); otherwise
 * that count or, below 32, a smaller power of two >= 2.  Fewer lanes change the order of a slice's FP32
 * sums (results within FP32 rounding, deterministic for a given choice).
 * bsgdtv_batch_autotune times the batch's count, half and a quarter of it
 * for each pass (keeping fewer lanes only when measurably faster) before its
 * FGP search. */
int bsgdtv_batch_set_pass_lanes(bsgdtv_batch_t h, int lanes_row, int lanes_col);

/* Copies slice b's x [cols] (FP32).  To the host: synchronises the stream. */
int bsgdtv_batch_get_slice_x(bsgdtv_batch_t h, int b, float *x, int out_on_device);

/* ------------------------------------------------------ packed batches
 * Several geometries (operators of one weight format, any sizes) with
 * `slices` slots each, whose epochs run together: each stage of an epoch --
 * the row pass r = y - A x, the column pass x^ = x + 2 mu A^T r_prev, the
 * transposes around the prox and every FGP launch -- is one kernel launch
 * over all parts (Algorithm 1 per slot, exactly as a batch slice of its
 * geometry), captured in one CUDA graph per epoch.  Uneven requests (images
 * of different sizes, angle and bin counts) thus share launches instead of
 * running one set per geometry.  Part k has its own y, lambdas and mu. */
typedef struct bsgdtv_packed_ctx *bsgdtv_packed_t;

/* Creates a packed batch of n_parts (1 .. 8) operators, `slices` slots each
 * (1 .. 4096), on `stream`.  Every part starts without data. */
int bsgdtv_packed_create(bsgdtv_packed_t *out, const bsgdtv_operator_t *ops, int n_parts, int slices,
                         void *stream);

/* Data of part `part`: as bsgdtv_batch_set_data for that part's geometry
 * (y [slices][rows of the part], lambdas [slices], mu for its A); restarts
 * the part's slots from x^0 = 0.  Every part needs data before a run. */
int bsgdtv_packed_set_part(bsgdtv_packed_t h, int part, const float *y, int y_on_device,
                           const double *lambdas, double mu);

/* Runs `epochs` epochs of every part (asynchronous on the handle's stream). */
int bsgdtv_packed_run(bsgdtv_packed_t h, int epochs, int fgp_iters);

/* x of part `part`, [slices][cols of the part] (synchronises for a host x). */
int bsgdtv_packed_get_x(bsgdtv_packed_t h, int part, float *x, int out_on_device);

/* Kernel launches in one epoch of the packed batch with fgp_iters FGP
 * iterations (builds the epoch graphs if needed). */
int bsgdtv_packed_launches_per_epoch(bsgdtv_packed_t h, int fgp_iters, int64_t *launches);

void bsgdtv_packed_destroy(bsgdtv_packed_t h);

/* ------------------------------------------------------ continuous batching
 * A reconstruction server: requests (projections of a registered geometry,
 * a TV weight and an epoch budget) are submitted at any time from any host
 * thread and run as slots of batch groups (bsgdtv_batch_*).  A geometry's A
 * is stored once (an operator) and shared by all its groups; a group is made
 * when a request finds no free slot, with a power-of-two number of slots
 * between 4 and the geometry's maximum, sized by the requests of that
 * geometry then waiting: a short queue gets small groups with short epochs
 * (low latency), a long queue large groups that read A once for many slices
 * (throughput).  A request is admitted into a free slot as soon as one
 * exists, also while its group runs: the worker posts it in the slot's
 * mailbox (host-mapped memory) and a slot scheduler kernel at the start of
 * every epoch admits it on the device, counts its epochs, and when its budget
 * is done writes its x to host memory and publishes a completion record.
 * Its x, r and FGP state stay on the device meanwhile.  One worker thread
 * inside the server keeps every busy group's stream fed with runs of epochs;
 * groups run on their own streams and overlap.  Admission keeps the device bytes (every A plus the
 * groups' vectors, bsgdtv_batch_device_bytes) within the budget, releasing
 * idle groups of other geometries first.  Every request runs Algorithm 1
 * exactly as a batch slice does: its result does not depend on the other
 * requests, bit for bit within groups of one size and within FP32 rounding
 * across sizes (the passes sum a slice's products in a grouping set by the
 * group's slice stride). */
typedef struct bsgdtv_server_ctx *bsgdtv_server_t;

/* Starts a server on the current device.  hbm_budget_bytes bounds the device
 * bytes of all geometries and groups; fgp_iters is the FGP iteration count of
 * every prox; max_tick_epochs caps the epochs of one run the worker enqueues
 * on a group (admissions and completions happen at every epoch boundary on
 * the device, whatever the run length). */
int bsgdtv_server_create(bsgdtv_server_t *out, int64_t hbm_budget_bytes, int fgp_iters,
                         int max_tick_epochs);

/* Stops the worker (requests still queued or running are abandoned), waits
 * for the device and frees everything.  NULL is ignored. */
void bsgdtv_server_destroy(bsgdtv_server_t s);

/* Registers a geometry: host CSR A as for bsgdtv_create_csr (validated and
 * uploaded once as an operator), the batch weight format
 * (bsgdtv_batch_create_csr_ex), the largest number of slots per group (0:
 * the largest power of two up to 32 for which a group's x and r, slots x
 * max(rows, cols) floats, fit in 64 MiB, so that the batch passes' gathers stay
 * in L2), the
 * step mu > 0 for this A (Theorem 1: mu < 1/(2 u_max), e.g. from
 * bsgdtv_estimate_umax) and how many groups of that size to create now
 * (prewarm, as far as the budget allows; the rest are made on demand).
 * Writes the geometry id.  Fails with BSGDTV_ERR_OOM if A and one smallest
 * group exceed what is left of the budget. */
int bsgdtv_server_add_geometry(bsgdtv_server_t s, int64_t rows, int64_t cols, int img_h, int img_w,
                               const int64_t *row_ptr, const int32_t *col_idx, const double *vals,
                               int format, int slots, double mu, int prewarm, int *geom_id);

/* Queues a request: y [rows of the geometry] (host FP32, copied), lambda >= 0,
 * epochs >= 1.  Writes its id.  Never blocks on the device. */
int bsgdtv_server_submit(bsgdtv_server_t s, int geom_id, const float *y, double lambda, int epochs,
                         int64_t *request_id);

/* Request state: 0 queued, 1 running, 2 done, 3 failed, 4 cancelled. */
int bsgdtv_server_poll(bsgdtv_server_t s, int64_t request_id, int *state);

/* Cancels a request that has not ended.  A queued one is cancelled at once;
 * a running one keeps its state "running" until the device's slot scheduler
 * sees the cancellation at its group's next epoch boundary and empties the
 * slot (its x is not returned).
 * bsgdtv_server_wait on a cancelled request returns BSGDTV_ERR_CANCELLED and
 * forgets it.  BSGDTV_ERR_STATE if the request is done, failed or cancelled
 * (state 2, 3 or 4); BSGDTV_ERR_INVALID_ARG for an unknown (or already waited-for)
 * id.  Cancellation is a serving feature; Algorithm 1 has no counterpart. */
int bsgdtv_server_cancel(bsgdtv_server_t s, int64_t request_id);

/* Waits up to timeout_s seconds (< 0: no limit) for the request; on success
 * copies its x [cols] to host memory x (may be NULL) and forgets the request.
 * times (may be NULL) receives [0] the latency from submit to x in host
 * memory and [1] the time spent queued, in seconds.  A failed request returns
 * its error code (and is forgotten); BSGDTV_ERR_TIMEOUT leaves it pending. */
int bsgdtv_server_wait(bsgdtv_server_t s, int64_t request_id, double timeout_s, float *x,
                       double *times);

/* Arms an idle group of the geometry (made if none exists and the budget
 * allows): one epoch is launched at once whose slot scheduler waits on the
 * device, polling the group's mailboxes, for up to wait_s seconds (0 <=
 * wait_s <= 1) for a request to be posted, so that a request submitted
 * meanwhile starts without waiting for a host launch.  Blocks until that
 * device-side wait has ended: BSGDTV_OK if a request arrived (it then runs as
 * usual), BSGDTV_ERR_TIMEOUT if the wait ran out with no request (the epoch
 * then ran on empty slots).  A serving feature; the paper has none. */
int bsgdtv_server_arm(bsgdtv_server_t s, int geom_id, double wait_s);

/* hold != 0: requests submitted from now on (and those queued) wait in the
 * queue without being admitted, while running ones carry on; hold = 0
 * admits them again, a burst of them together (which lets packing see every
 * geometry of the burst at once).  A serving feature; the paper has none. */
int bsgdtv_server_hold(bsgdtv_server_t s, int hold);

/* Packing of uneven requests: a group the server makes for a geometry also
 * takes, as further parts of one packed batch (bsgdtv_packed_*), up to
 * max_parts - 1 other geometries that have requests waiting and no free
 * slot, need the same slot count, share the weight format and whose
 * operators hold within cost_ratio times the nonzeros of each other; every
 * epoch stage of the group is then one launch for all of them.  max_parts = 1
 * (the default) packs nothing.  Applies to groups made afterwards. */
int bsgdtv_server_set_packing(bsgdtv_server_t s, int max_parts, double cost_ratio);

/* by_size != 0 (the default): each group runs on a stream whose priority is
 * one step higher for every factor of 16 by which its operator has fewer
 * nonzeros than the largest registered one, within the device's priority
 * range, so that when SMs free up the short kernels of much smaller images are
 * scheduled before the long kernels of large ones (running kernels are not
 * preempted; results do not change); geometries within a factor of 16 of each
 * other share a priority.  0: every group at the default priority.  Applies to
 * groups made afterwards. */
int bsgdtv_server_set_priority(bsgdtv_server_t s, int by_size);

/* stats [18]: submitted, completed, failed, queued, running, groups, device
 * bytes in use (operators and groups), most requests running at once, runs
 * of epochs launched, epochs run by groups, slice-epochs of requests, groups
 * created, cancelled, armed epochs, armed waits that timed out, packed groups
 * created (more than one geometry), most geometries in one group, kernel
 * launches per epoch of the last packed group made. */
int bsgdtv_server_stats(bsgdtv_server_t s, int64_t *stats);

#ifdef __cplusplus
}
#endif

#endif /* BSGDTV_H */
