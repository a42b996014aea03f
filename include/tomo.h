/*
 * tomo.h -- C ABI of the B300 sparse-matrix tomography library (libtomo.so).
 *
 * The library builds the parallel-beam projector A of Sec. 2 ("Tomography":
 * the projection P_theta(p) is the integral of u along the line
 * x cos(theta) + y sin(theta) = p) as a sparse ray-by-pixel matrix, stores its
 * transpose explicitly (Sec. 3.1: matrix and transpose are kept as two separate
 * sparse matrices), and applies both to batches of slices (Sec. 3: SpMV /
 * SpMM over a stack of sinograms or tomograms) inside SIRT and CGLS (Sec. 2.1).
 *
 * Conventions shared by every call
 *   - Pixel (ix, iy) is the unit square centred at x = ix + 1/2 - n_x/2,
 *     y = iy + 1/2 - n_y/2; column j = iy*n_x + ix.  A tomogram batch is
 *     (n_z, n_y, n_x) floats, x fastest.
 *   - Row i = m*n_p + k is the ray of angle theta_m through the centre of
 *     detector bin k, p_k = k + 1/2 - c.  A sinogram batch is
 *     (n_z, n_theta, n_p) floats.
 *   - A[i, j] is the chord length of ray i through pixel j: with
 *     a = max(|cos|,|sin|), e = min(|cos|,|sin|), h = (a+e)/2 and
 *     delta = |p_k - (x cos + y sin)|, the pixel is hit iff delta < h and the
 *     length is 1/a when delta <= (a-e)/2, else (h - delta)/(a e).  Membership
 *     and lengths are decided in IEEE FP64 (no fused multiply-add), so the
 *     structure is reproducible bit for bit on any IEEE machine.
 *   - Every float pointer passed to a compute call is a DEVICE pointer on the
 *     current CUDA device, 16-byte aligned, owned by the caller and never
 *     freed by the library.  Host pointers are only used where stated.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Compute calls are asynchronous on that stream unless stated.
 *   - Errors are return codes; nothing throws across this boundary.  Invalid
 *     arguments are rejected before any work is queued.  CUDA launch errors
 *     are reported as TOMO_ERR_CUDA.
 */
#ifndef TOMO_H
#define TOMO_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TOMO_API __attribute__((visibility("default")))
#else
#define TOMO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TOMO_OK = 0,
  TOMO_ERR_INVALID_ARG = 1,
  TOMO_ERR_OOM = 2,
  TOMO_ERR_CUDA = 3,
  TOMO_ERR_TIMEOUT = 4,
  TOMO_ERR_UNSUPPORTED = 5,
  TOMO_ERR_NUMERIC = 6,
  TOMO_ERR_IO = 7
} tomo_status;

typedef enum { TOMO_F32 = 0, TOMO_BF16 = 1, TOMO_F16 = 2 } tomo_dtype;

typedef enum {
  TOMO_SLICE_MAJOR = 0, /* (n_z, rows): one contiguous slice after another      */
  TOMO_INTERLEAVED = 1  /* (rows, n_z): the n_z values of one row are adjacent */
} tomo_layout;

/* Acquisition geometry (Sec. 2).  `angles` is a HOST array of n_theta radians
 * (copied during the call; NULL selects theta_m = m*pi/n_theta).  `center` is
 * the detector coordinate of the rotation axis in bins (Sec. 3: c = n_p/2 when
 * the axis projects onto the central detector column); NaN selects n_p/2. */
typedef struct {
  int32_t n_x, n_y, n_p, n_theta;
  const double *angles;
  double center;
} tomo_geometry;

/* Discretisation of the line integral of Sec. 2 over a pixel image. */
typedef enum {
  TOMO_MODEL_LINE = 0, /* chord length of the line x cos + y sin = p_k through the pixel square */
  TOMO_MODEL_STRIP = 1 /* area of the pixel square inside the strip |x cos + y sin - p_k| < 1/2
                          (the line integral averaged over a detector bin of unit width);
                          about 1.7x the entries of the line model, exact per-angle mass */
} tomo_model;

/* Build options.  values: TOMO_F32 builds the FP32 operands (canonical CSR and
 * the SELL-32 form the kernels stream).  TOMO_BF16 / TOMO_F16 also build the
 * 16-bit encoding (16-bit values scaled per angle so a full chord is exactly
 * 1.0, uint16 column offsets against a 32-bit base per 16 entries of a row)
 * that compute calls use when exec opts select TOMO_FMT_SELL16. */
typedef struct {
  int32_t values;        /* tomo_dtype */
  int32_t no_fp32_sell;  /* non-zero: skip the FP32 SELL-32 pair (saves ~8.4 B/nnz per operand when
                            only the 16-bit or the CSR form will be streamed) */
  int32_t drop_csr;      /* non-zero: free the CSR pair once the SELL forms are built (saves 8 B/nnz
                            per operand); export calls and TOMO_FMT_CSR then report UNSUPPORTED.
                            Needs at least one SELL form. */
  int32_t model;         /* tomo_model (default TOMO_MODEL_LINE) */
  int32_t col_blocks;    /* 16-bit values only: store the 16-bit A as this many column bands (bands of
                            consecutive image rows, each its own 16-bit SELL-32 matrix) instead of one;
                            a projection then runs one pass per band and adds the bands' partial sums
                            in a workspace buffer, so that each pass gathers only its band of the image
                            (which can stay in L2 when the whole image stack cannot).  0 (default):
                            enough bands that one band of a 16-slice FP32 image batch fits in 48 MB
                            (1 up to about 886 x 886 pixels); 1: one band; at most min(64, n_y).
                            tomo_cgls_batched runs a banded A one band at a time (a grid barrier
                            between bands). */
  int32_t no_at_tiles;   /* 16-bit values only.  0 (default): also store the 16-bit A^T in image tiles of
                            16 x 16 pixels (about 4.7 B/nnz more), for the SIRT / CGLS passes at batch
                            width 16 that stage each tile's detector window, 8 angles at a time, in
                            shared memory (order 3 of tomo_exec_opts).  Non-zero: do not build it. */
  int32_t a_ray_order;   /* 16-bit values only.  0 (default): when n_theta is even and n_p a multiple of 4,
                            store the 16-bit A's rows in pair order: each 8 consecutive rows are the
                            rays of 2 adjacent angles x 4 adjacent bins, which one warp gathers together
                            at batch width 16 (their image rows coincide more often in L1 than those of
                            8 bins at one angle).  Same results, bit for bit.  Non-zero: rays in their
                            natural order. */
  int32_t reserved[1];
} tomo_matrix_opts;

/* Device time of the kernels one call launched, filled when a call is given
 * a tomo_exec_opts with `timing` set.  Kinds: [0] SpMM with A (projection
 * passes), [1] SpMM with A^T (backprojection passes), [2] every other kernel
 * (layout changes, solver vector and scalar updates), [3] unused. */
typedef struct {
  double ms[4];         /* summed device milliseconds per kind */
  int64_t launches[4];  /* kernels launched per kind */
} tomo_timing;

/* Matrix storage a compute call streams. */
typedef enum {
  TOMO_FMT_SELL = 0,   /* FP32 values, SELL-32 chunks, 128-bit entry loads (default) */
  TOMO_FMT_SELL16 = 1, /* 16-bit values + 16-bit column offsets (needs a 16-bit build) */
  TOMO_FMT_CSR = 2,    /* FP32 CSR as exported: CSR-vector SpMV for widths 1-2, the plain comparator */
  TOMO_FMT_AUTO = 3    /* the format tomo_autotune chose for this slice count (else TOMO_FMT_SELL) */
} tomo_format;

/* Per-call execution options (pointer may be NULL = defaults). */
typedef struct {
  int32_t batch_width; /* slices per SpMM pass: 0 = the width tomo_autotune chose for this slice count,
                          else the library default; or one of 1,2,4,8,16,32,64 */
  int32_t use_graph;   /* SIRT/CGLS: replay one captured iteration as a CUDA graph (default 1) */
  int32_t format;      /* tomo_format of the matrix operands (default TOMO_FMT_SELL) */
  float timeout_s;     /* tomo_cgls_batched: limit of each grid-barrier wait in seconds (0 = 10) */
  tomo_timing *timing; /* non-NULL: bracket every launch with CUDA events on the call's stream,
                          launch without graphs, synchronise the stream before returning and
                          ADD the measured times and counts into *timing */
  int32_t test_flags;  /* test hook, 0 in normal use.  bit 0: in tomo_cgls_batched one block of
                          the persistent launch never arrives at a grid barrier, so the others
                          wait out timeout_s and the call returns TOMO_ERR_TIMEOUT */
  int32_t async;       /* tomo_cgls_batched: non-zero returns once the launch is queued, without
                          synchronising; the launch's device status then goes to the stream's
                          status word (tomo_stream_status).  Sinograms, tomograms, states and
                          the workspace must stay valid until the stream passes the launch. */
  int32_t recompute_fp32; /* tomo_cgls / tomo_cgls_resume with TOMO_FMT_SELL16: non-zero computes
                          the periodic residual r = b - A x with the FP32 values of A (the FP32
                          SELL form when built, else CSR) instead of the 16-bit ones */
  int32_t order;       /* order in which the SELL A^T passes visit their rows (pixels): 0 = auto
                          (3 where it applies, else image tiles when the gathered sinogram batch
                          exceeds 64 MB, else row order), 1 = row order, 2 = image tiles (blocks of
                          8 image rows, tiles of 128 rows, so a block's rays share sinogram rows in
                          L1 and a tile's stay in L2), 3 = staged tiles: the SIRT / CGLS A^T passes
                          with TOMO_FMT_SELL16 at batch width 16 on a matrix with the tiled 16-bit
                          A^T (tomo_matrix_opts.no_at_tiles = 0) stream it, one block per 16 x 16
                          pixel tile, gathering from the tile's detector window staged in shared
                          memory (other passes keep order 2).  The results are the same bits
                          either way.  After tomo_autotune for this slice count, 0 selects the
                          tuned order. */
  int32_t blocks_per_sm; /* resident blocks per SM the SpMM launches use: 0 = all that fit (or the
                          tuned count after tomo_autotune for this slice count), else at most this
                          many.  The results are the same bits either way. */
  int32_t reserved[3];
} tomo_exec_opts;

typedef struct tomo_matrix tomo_matrix; /* opaque, immutable after build */

typedef struct {
  int64_t rows, cols, nnz;
  int64_t bytes_f32;   /* device bytes of the FP32 CSR pair (A and A^T) */
  int64_t bytes_lp;    /* device bytes of the 16-bit pair (0 if not built) */
  int64_t max_row_len, max_col_len;
  int32_t lp_dtype;    /* tomo_dtype of the 16-bit values (TOMO_F32 if none) */
  int32_t at_tiles;    /* non-zero when the 16-bit A^T is also stored in image tiles (order 3) */
} tomo_matrix_info_t;

/* Operations that need scratch memory; see tomo_workspace_size. */
typedef enum {
  TOMO_OP_PROJECT = 0,
  TOMO_OP_BACKPROJECT = 1,
  TOMO_OP_SIRT = 2,
  TOMO_OP_CGLS = 3,
  TOMO_OP_SIRT_BB = 4,
  TOMO_OP_RESIDUAL = 5
} tomo_op;

/* Build A and A^T on the current device (Sec. 3.1: entries generated from the
 * geometry, zero / out-of-range entries dropped, CSR sorted by row and by
 * column; the transpose is stored separately).  A is rows = n_theta*n_p by
 * cols = n_x*n_y with int64 row pointers, int32 columns ascending within each
 * row and FP32 values (FP64 chord lengths rounded to nearest).  Also computes
 * the SIRT normalisers R_i = 1/sum_j A_ij and C_j = 1/sum_i A_ij (0 where the
 * sum is 0).  Synchronises `stream` (nnz must be known to allocate).
 * Errors: INVALID_ARG for non-positive sizes, non-finite angles or center,
 * or sizes beyond int32 columns; OOM if the device cannot hold the matrices
 * (nothing is left allocated); CUDA on launch failures. */
TOMO_API tomo_status tomo_build_matrix(const tomo_geometry *geom, const tomo_matrix_opts *opts,
                                       void *stream, tomo_matrix **out);

/* Free every device buffer of the handle.  NULL is accepted. */
TOMO_API tomo_status tomo_matrix_destroy(tomo_matrix *A);

/* Sizes of the handle (host struct filled synchronously). */
TOMO_API tomo_status tomo_matrix_info(const tomo_matrix *A, tomo_matrix_info_t *info);

/* Copy rows [row_begin, row_end) of A (transpose = 0) or of A^T (transpose = 1)
 * to HOST buffers: row_ptr gets row_end-row_begin+1 offsets relative to the
 * first exported row, col / val the entries (capacity `cap` entries; the call
 * fails with INVALID_ARG when the range holds more, after filling row_ptr).
 * Synchronous.  For parity checks of the stored structure. */
TOMO_API tomo_status tomo_matrix_export_rows(const tomo_matrix *A, int32_t transpose, int64_t row_begin,
                                             int64_t row_end, int64_t *row_ptr, int32_t *col, float *val,
                                             int64_t cap);

/* Copy the whole CSR form of A (transpose = 0) or of its stored transpose
 * (transpose = 1) to HOST buffers: row_ptr (rows + 1 offsets), col and val
 * (nnz entries each; sizes from tomo_matrix_info).  Enqueued on `stream` and
 * synchronised before return.  UNSUPPORTED when the handle dropped its CSR
 * form.  For parity checks of the stored structure. */
TOMO_API tomo_status tomo_matrix_export_csr(const tomo_matrix *A, int32_t transpose, int64_t *row_ptr, int32_t *col,
                                            float *val, void *stream);

/* Copy the SIRT normalisers to HOST buffers (R: rows floats, C: cols floats;
 * either may be NULL).  Synchronous. */
TOMO_API tomo_status tomo_matrix_export_norms(const tomo_matrix *A, float *R, float *C);

/* Bytes of scratch a call needs for n_z slices with the given options.  A call
 * given workspace = NULL allocates this much itself (stream-ordered) and frees
 * it before returning. */
TOMO_API tomo_status tomo_workspace_size(const tomo_matrix *A, int32_t op, int32_t n_z,
                                         const tomo_exec_opts *opts, size_t *bytes);

/* Forward projection y = A x for n_z slices (Sec. 2 Radon transform, applied as
 * SpMM with the slices as right-hand sides; Sec. 3).  x: n_z tomograms, y: n_z
 * sinograms, both in `layout`.  TOMO_INTERLEAVED requires n_z to be one of
 * 1,2,4,8,16,32,64.  Errors: INVALID_ARG (NULL / unaligned pointers, n_z < 1),
 * UNSUPPORTED (interleaved n_z not a supported width, or TOMO_FMT_SELL16 on a
 * matrix built without the 16-bit encoding). */
TOMO_API tomo_status tomo_project(const tomo_matrix *A, const float *x, float *y, int32_t n_z, int32_t layout,
                                  const tomo_exec_opts *opts, void *workspace, size_t workspace_bytes,
                                  void *stream);

/* Backprojection x = A^T y with the stored transpose (no atomics). */
TOMO_API tomo_status tomo_backproject(const tomo_matrix *A, const float *y, float *x, int32_t n_z,
                                      int32_t layout, const tomo_exec_opts *opts, void *workspace,
                                      size_t workspace_bytes, void *stream);

/* SIRT (Sec. 2.1), classical form: x <- x + lambda * C o A^T (R o (b - A x)),
 * `iters` times, for n_z independent slices.  sino: (n_z, n_theta, n_p);
 * x: (n_z, n_y, n_x), holds the start on entry and the result on return. */
TOMO_API tomo_status tomo_sirt(const tomo_matrix *A, const float *sino, float *x, int32_t n_z, int32_t iters,
                               float lambda, const tomo_exec_opts *opts, void *workspace,
                               size_t workspace_bytes, void *stream);

/* CGLS (Sec. 2.1) for min ||A x - b|| per slice from x0 = 0: vectors FP32,
 * inner products, norms and the step scalars alpha / beta in FP64 on the
 * device.  Every `recompute_every` iterations (0 = never) the residual is
 * recomputed as r = b - A x (with the format's own values, or with the FP32
 * ones when opts->recompute_fp32 is set).  A slice whose ||s||^2 or ||q||^2 reaches 0 stops
 * changing.  resnorm_hist (DEVICE, nullable) receives ||r|| per iteration and
 * slice, laid out (iters, n_z).  x: (n_z, n_y, n_x) output. */
TOMO_API tomo_status tomo_cgls(const tomo_matrix *A, const float *sino, float *x, int32_t n_z, int32_t iters,
                               int32_t recompute_every, double *resnorm_hist, const tomo_exec_opts *opts,
                               void *workspace, size_t workspace_bytes, void *stream);

/* The data fit ||b - A x|| of every slice (the objective CGLS minimises,
 * Sec. 2.1) with FP64 accumulation: the product of an FP32 value and an FP32
 * operand is exact in FP64 and every sum is FP64, so the result is the data
 * fit of the FP32-valued operator to about 1e-15 relative, whatever the row
 * length (an FP32 SpMM loses ~1e-6 of ||b|| to rounding, which is a large part
 * of a small residual).  For stopping rules and for comparing solves of
 * different precision at equal data fit.  sino (n_z, n_theta, n_p) and x
 * (n_z, n_y, n_x) are DEVICE, slice-major; norms (DEVICE, 8-byte aligned)
 * receives n_z doubles.  Uses the FP32 CSR form of A (UNSUPPORTED when the
 * handle dropped it).  Workspace: tomo_workspace_size with TOMO_OP_RESIDUAL
 * (NULL: allocated stream-ordered by the call).  Deterministic: the sums run
 * in a fixed order. */
TOMO_API tomo_status tomo_residual_norm(const tomo_matrix *A, const float *sino, const float *x, int32_t n_z,
                                        double *norms, void *workspace, size_t workspace_bytes, void *stream);

/* SIRT exactly as tomo_sirt, for callers that cannot allocate GPU memory at
 * all.  The paper has no counterpart; this entry point exists for programs
 * that reconstruct inside a fixed memory budget, such as a reconstruction
 * loop embedded in a detector's acquisition software: cudaMalloc / cudaFree
 * may synchronise the device (stalling the streams that move frames) and may
 * fail under memory pressure in the middle of a scan, so such a caller can
 * neither pass a workspace it allocated nor let the library allocate one.
 *
 * The call allocates nothing.  Its scratch is a 16 MiB array compiled into
 * the library; every GPU that loads the library reserves it until the process
 * exits.  The call looks up that array's device address on the current
 * device each time (a device reset may move it), except while `stream` is
 * being captured, when it takes the address an earlier call on that device
 * found: make the first call on a device before any stream capture.  Batch width
 * is chosen internally (the widest of 16, 8, 4, 2, 1, not above n_z, whose
 * scratch fits); a geometry whose residual alone exceeds 16 MiB (more than
 * 4,194,304 rays) is rejected with TOMO_ERR_INVALID_ARG and a message giving
 * the bytes it would need.  All calls share the one array: calls that can
 * overlap on the GPU (different streams, or different host threads) race on
 * it and must be serialised by the caller.  Nothing in the array has to start
 * at zero; every word a call reads it has written first.  Arguments as for
 * tomo_sirt; kernels are launched on `stream` without CUDA graphs. */
TOMO_API tomo_status tomo_sirt_noalloc(const tomo_matrix *A, const float *sino, float *x, int32_t n_z,
                                       int32_t iters, float lambda, void *stream);

/* CGLS state of n_z slices (checkpoint / resume), caller-owned DEVICE
 * buffers, slice-major: r (n_z, rows) = b - A x, p (n_z, cols) the search
 * direction, gamma (n_z) = ||A^T r||^2 in FP64, frozen (n_z) 1 for a slice
 * that has converged (gamma or ||A p||^2 reached 0), else 0.  r and p
 * 16-byte aligned. */
typedef struct {
  float *r;
  float *p;
  double *gamma;
  int32_t *frozen;
} tomo_cgls_state;

/* State of the BB-step SIRT of n_z slices, caller-owned DEVICE buffers,
 * slice-major: g (n_z, cols) = A^T P^T P (b - A x) of the last step (16-byte
 * aligned), alpha (n_z) the last step length (FP64), frozen (n_z) 1 for a
 * slice whose BB step broke down (<s,s> or <s,y> not positive: converged).
 * alpha = 0 with frozen = 0 means "no step taken yet". */
typedef struct {
  float *g;
  double *alpha;
  int32_t *frozen;
} tomo_bb_state;

/* SIRT with Hamming preconditioning and the Barzilai-Borwein step (Sec. 3.1:
 * the paper's SIRT), minimising ||P (A x - b)||^2 per slice with the
 * preconditioner P = F^dagger D^(1/2) F of Sec. 2.1 applied along the
 * detector of every projection.  D is the N-point DFT of the sampled
 * band-limited ramp (1/4 at 0, -1/(pi n)^2 at odd n) times the Hamming window
 * 0.54 + 0.46 cos(2 pi f), N the smallest power of two >= 2 n_p; P^T P runs as
 * the exact Toeplitz product of those taps over the n_p bins (no FFT).
 * Iteration k, per slice: r = b - A x (||r|| -> resnorm_hist[k * n_z + z],
 * DEVICE, nullable); g = A^T P^T P r; alpha = first_step for a slice's first
 * step (first_step <= 0 selects pi / n_theta, which makes the first iterate
 * from x = 0 the filtered backprojection, Sec. 2.1), else the BB step
 * <s,s>/<s,y> with s the last step and y the change of -g, in FP64; a slice
 * whose <s,s> or <s,y> is not positive is frozen; x += alpha g.
 * x (n_z, n_y, n_x) is the starting iterate on entry (zero it for x0 = 0) and
 * the result on return.  in (nullable): continue from a saved state (x the
 * matching iterate); out (nullable): the state after the last iteration.
 * Workspace: tomo_workspace_size with TOMO_OP_SIRT_BB. */
TOMO_API tomo_status tomo_sirt_bb(const tomo_matrix *A, const float *sino, float *x, int32_t n_z, int32_t iters,
                                  double first_step, double *resnorm_hist, const tomo_bb_state *in,
                                  tomo_bb_state *out, const tomo_exec_opts *opts, void *workspace,
                                  size_t workspace_bytes, void *stream);

/* One reconstruction request of tomo_cgls_batched: DEVICE buffers sino
 * (n_z, n_theta, n_p) and x (n_z, n_y, n_x), both 16-byte aligned, on the
 * geometry of A; resnorm_hist (DEVICE, nullable) receives ||r|| as
 * (iters, n_z).  state_in (nullable): continue from that CGLS state, with x
 * holding the matching iterate on entry; state_out (nullable): receives the
 * state after the last iteration (see tomo_cgls_resume). */
typedef struct {
  const tomo_matrix *A;
  const float *sino;
  float *x;
  int32_t n_z;
  int32_t reserved;
  double *resnorm_hist;
  const tomo_cgls_state *state_in;
  tomo_cgls_state *state_out;
} tomo_request;

/* CGLS (Sec. 2.1) for many requests of uneven size in ONE persistent launch
 * (Sec. 3.1 splits uneven slice counts into chunks; here requests sharing a
 * geometry handle are packed batch_width slices at a time).  Every slice runs
 * `iters` iterations from x0 = 0 as in tomo_cgls (no residual recompute).
 * opts: batch_width 4, 8, 16 (default) or 32; format TOMO_FMT_SELL (default)
 * or TOMO_FMT_SELL16 (every matrix built with the same 16-bit type);
 * timeout_s bounds each grid-barrier wait.  All matrices on one device.  With
 * 16-bit values the A^T phases gather the residual pre-scaled by 1/a(theta),
 * and a matrix whose 16-bit A is stored as column bands runs its A phase band
 * by band.  Inside a phase the blocks take (batch, 8 row groups) work items in
 * list order.  The launch is cooperative (every block resident), the barriers
 * are bounded: a
 * wait that runs out stops every block and the call returns TOMO_ERR_TIMEOUT.
 * Workspace as tomo_cgls_batched_workspace reports (NULL: allocated by the
 * call, stream-ordered).  Synchronises `stream` and returns the launch's
 * status, unless opts->async is set: then it returns after queueing and the
 * status is read later with tomo_stream_status. */
TOMO_API tomo_status tomo_cgls_batched(const tomo_request *reqs, int32_t n_reqs, int32_t iters,
                                       const tomo_exec_opts *opts, void *workspace, size_t workspace_bytes,
                                       void *stream);

/* Workspace bytes tomo_cgls_batched needs for these requests and options. */
TOMO_API tomo_status tomo_cgls_batched_workspace(const tomo_request *reqs, int32_t n_reqs,
                                                 const tomo_exec_opts *opts, size_t *bytes);

/* One timed candidate of tomo_autotune. */
typedef struct {
  int32_t batch_width, format;
  int32_t order;             /* row-group order of the A^T pass (1 rows, 2 image tiles, 3 staged tiles) */
  int32_t blocks_per_sm;     /* resident blocks per SM (0 = all that fit) */
  double ms_per_iter;        /* one SIRT iteration (A pass + A^T pass) over one batch of batch_width slices */
  double slice_iters_per_s;  /* for n_z slices: n_z / (ceil(n_z / batch_width) * ms_per_iter) */
} tomo_tune_entry;

/* Autotuner of the SpMM launch shape.  The paper picks no such parameters; it
 * relies on library SpMV.  Times one SIRT iteration (the A pass with the
 * residual epilogue and the A^T pass with the update epilogue, the same
 * kernels tomo_sirt replays) on device scratch.  Stage 1: every batch width
 * 1..64 not above n_z rounded up to a power of two (the width fixes the row
 * block of a warp: 32 / max(1, width / 4) rows), every format (TOMO_FMT_SELL,
 * TOMO_FMT_CSR and, when allow_16bit is non-zero and the matrix has a 16-bit
 * encoding, TOMO_FMT_SELL16; allow_16bit = 2 searches TOMO_FMT_SELL16 alone),
 * and for the SELL formats both row-group orders
 * of the A^T pass (rows, image tiles).  Stage 2: the best stage-1 shape with
 * fewer resident blocks per SM (all that fit minus 1 and minus 2).  Writes up
 * to `cap` candidates to `table` (nullable) and their count to *n_table,
 * returns the fastest in *best (batch_width, format, order, blocks_per_sm)
 * with its rate in *rate, and remembers it in the handle for later calls with
 * that n_z (up to 8 slice counts) that pass batch_width = 0, format =
 * TOMO_FMT_AUTO, order = 0 or blocks_per_sm = 0.  Allocates its scratch with
 * cudaMalloc and synchronises `stream`.  Not to be called while other calls
 * on the same handle are being queued from another thread. */
TOMO_API tomo_status tomo_autotune(tomo_matrix *A, int32_t n_z, int32_t allow_16bit, tomo_exec_opts *best,
                                   double *rate, tomo_tune_entry *table, int32_t cap, int32_t *n_table,
                                   void *stream);

/* CGLS (Sec. 2.1) continued from a saved state: `in` (nullable) holds the
 * state after some iterations and x (n_z, n_y, n_x) the matching iterate;
 * with in = NULL the call starts from x0 = 0 exactly as tomo_cgls.  `out`
 * (nullable) receives the state after the last iteration.  Iteration
 * numbering (the recompute cadence and the rows of resnorm_hist) restarts at
 * 0 in every call, so k iterations then a resume for m give the same bits as
 * k + m iterations when recompute_every divides k (or is 0). */
TOMO_API tomo_status tomo_cgls_resume(const tomo_matrix *A, const float *sino, float *x, int32_t n_z,
                                      int32_t iters, int32_t recompute_every, double *resnorm_hist,
                                      const tomo_cgls_state *in, tomo_cgls_state *out,
                                      const tomo_exec_opts *opts, void *workspace, size_t workspace_bytes,
                                      void *stream);

/* ---------------------------------------------------------------------------
 * The Fubini-Radon transform (Sec. 3, Eq. 2): the projector computed through
 * the Fourier slice theorem.  Radon(u) = F1^-1 S^H F2 (k* o u): deapodize
 * (k* = 1 / the Kaiser-Bessel window's transform), zero-pad the n x n image to
 * a 2n x 2n grid, 2D FFT, interpolate the spectrum onto the polar samples
 * (theta_m, w_q = (q - floor(n_p/2)) / n_p) with the sparse gridding matrix S
 * (Kaiser-Bessel window of kw x kw grid points, shape beta = pi sqrt((kw/2)^2
 * 1.5^2 - 0.8)), 1D inverse FFT along each radial line, real part.  It
 * approximates, to the gridding error (about 3e-6 relative at kw = 6), the
 * exact transform R[u](m,k) = Re((1/n_p) sum_q e^{2 pi i w_q p_k}
 * sum_j u_j e^{-2 pi i w_q (x_j cos theta_m + y_j sin theta_m)}) with the pixel
 * and bin coordinates of the line model.  S is real; the paper's phase ramp
 * and FFT shifts are applied as diagonal phases beside the FFTs.  The 2D
 * FFTs are hand-written register FFTs when 2n is a power of two up to 2048
 * (cuFFT otherwise), the 1D ones cuFFT calls; S and its stored transpose are
 * built on the device.
 * ------------------------------------------------------------------------- */
typedef struct tomo_fubini tomo_fubini; /* holds S, S^T, cuFFT plans and scratch: one call at a time */

/* Build the operator for geom (n_x == n_y required; angles and center as for
 * tomo_build_matrix) with a window of kw grid points (even, 2..16; 6 gives
 * about 3e-6, 8 about 2e-8 relative error).  Synchronises `stream`. */
TOMO_API tomo_status tomo_fubini_create(const tomo_geometry *geom, int32_t kw, void *stream, tomo_fubini **out);

/* Free every device buffer and plan of the handle.  NULL is accepted. */
TOMO_API tomo_status tomo_fubini_destroy(tomo_fubini *F);

/* y (n_z, n_theta, n_p) = Radon(x) for x (n_z, n, n); DEVICE buffers,
 * slice-major.  Calls on one handle must not overlap (shared scratch). */
TOMO_API tomo_status tomo_fubini_project(tomo_fubini *F, const float *x, float *y, int32_t n_z, void *stream);

/* x = the exact adjoint of tomo_fubini_project applied to y (filter 0), or the
 * filtered backprojection iRadon (filter 1: the adjoint with the ramp density
 * |w_q| on the polar samples, the DC sample weighted 1/(4 n_p), and the
 * angular weight pi/n_theta; Sec. 3's D), or the same with the density times
 * the Hamming window 0.54 + 0.46 cos(2 pi w_q) (filter 2). */
TOMO_API tomo_status tomo_fubini_backproject(tomo_fubini *F, const float *y, float *x, int32_t n_z, int32_t filter,
                                             void *stream);

/* The paper's SIRT (Sec. 3.1: Hamming preconditioning, BB step) on this
 * operator: per slice from x = 0, r = b - Radon(x) (||r|| -> resnorm_hist
 * [k * n_z + z], DEVICE, nullable), g = iRadon_Hamming(r) (filter 2), x += alpha
 * g with alpha = 1 on the first step (x_1 = the filtered backprojection of b)
 * and the BB1 step <s,s>/<s,y> after it (FP64 per slice; a slice whose <s,s>
 * or <s,y> is not positive is frozen).  sino (n_z, n_theta, n_p) and x
 * (n_z, n, n) DEVICE.  Scratch is allocated stream-ordered on `stream`. */
TOMO_API tomo_status tomo_fubini_sirt_bb(tomo_fubini *F, const float *sino, float *x, int32_t n_z, int32_t iters,
                                         double *resnorm_hist, void *stream);

/* The TV prior of the model-based objective (Sec. 2.1), value and gradient in
 * one pass: per slice s of x (n_z, n_y, n_x), DEVICE, slice-major,
 *   loss[s] = sum_{iy,ix} sqrt(Dx^2 + Dy^2 + eps^2)   (FP64, DEVICE, n_z values)
 * with forward differences Dx = x[iy][ix+1] - x[iy][ix], Dy = x[iy+1][ix] -
 * x[iy][ix] (0 on the last column / row), and grad (same shape as x, DEVICE)
 * = d loss[s] / d x_s.  The value is summed in FP64 in a fixed order
 * (deterministic).  eps > 0 with eps^2 a normal FP32 number (eps >= 1.1e-19);
 * n_z <= 65535. */
TOMO_API tomo_status tomo_tv(const float *x, int32_t n_z, int32_t n_y, int32_t n_x, float eps, double *loss,
                             float *grad, void *stream);

/* The normal operator in one step (the Toeplitz route of the outlook, Sec. 5):
 * y = N x, N = R^T W R for the EXACT transform R above and the sinogram weight
 * W of the exact adjoint (filter 0), of iRadon with the ramp density (1) or
 * with the Hamming-windowed density (2) -- the same filters as
 * tomo_fubini_backproject.  For real images
 *   N[j,l] = t(x_j - x_l) + h(x_j + x_l),
 *   t(d) = kappa sum_m sum_q nu_q cos(2 pi w_q (d . theta_m)),
 *   h(s) = kappa (D_q0/2) sum_m cos(2 pi (1/2 - c) - pi (s . theta_m)),
 * (kappa = 1/n_p for filter 0, pi/(n_theta n_p) otherwise; D_q the density,
 * nu_q = D_q except nu_q0 = D_q0/2 and h = 0 unless n_p is even, q0 being the
 * unpaired sample w = -1/2), applied as a circular convolution on the 2n x 2n
 * grid: an FP32 FFT of the padded image, one pointwise product, the inverse FFT
 * (hand-written register FFTs when 2n is a power of two up to 2048, cuFFT
 * otherwise);
 * no gridding, no 1D transforms.  It agrees with
 * tomo_fubini_backproject(tomo_fubini_project(x)) to the gridding error.  The
 * first call per filter sums the taps in FP64 on the device and transforms
 * them (O(n^2 n_theta n_p) work, synchronises `stream`).  x, y (n_z, n, n)
 * DEVICE, slice-major, not overlapping. */
TOMO_API tomo_status tomo_fubini_normal(tomo_fubini *F, const float *x, float *y, int32_t n_z, int32_t filter,
                                        void *stream);

/* The paper's SIRT of tomo_fubini_sirt_bb with the normal operator: per slice
 * c = iRadon_Hamming(sino) once (gridded), then g_k = c - N x_k (filter 2;
 * ||g_k|| -> gradnorm_hist[k * n_z + z], DEVICE, nullable), x += alpha g with
 * alpha = 1 first and the BB1 step after it, as there.  One convolution per
 * iteration instead of a projection and a backprojection.  n_z <= 65535.
 * Scratch is allocated stream-ordered on `stream`. */
TOMO_API tomo_status tomo_fubini_sirt_bb_normal(tomo_fubini *F, const float *sino, float *x, int32_t n_z,
                                                int32_t iters, double *gradnorm_hist, void *stream);

/* Device-side status of `stream` (a stream of the CURRENT device; NULL = the
 * legacy default stream).  Calls queued without synchronising (tomo_cgls_batched
 * with opts->async) record the status of their bounded waits in one status
 * word per (device, stream) that the library keeps.  This call synchronises
 * the stream, returns the first non-OK status recorded since the previous
 * tomo_stream_status on it (TOMO_ERR_TIMEOUT: a grid-barrier wait ran out and
 * the launch stopped early, its outputs incomplete) and resets the word; it
 * returns TOMO_ERR_CUDA when the synchronisation itself reports an error.
 * The word is allocated (4 bytes) on first use and kept until process exit. */
TOMO_API tomo_status tomo_stream_status(void *stream);

/* Human-readable name of a status code (static string). */
TOMO_API const char *tomo_status_string(tomo_status s);

/* Message of the last failure on the calling thread (static per-thread buffer). */
TOMO_API const char *tomo_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TOMO_H */
