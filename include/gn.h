/*
 * gn.h -- C ABI of the GB300 generalized Nystrom (GN) library.
 *
 * Generalized Nystrom (Nakatsukasa, arXiv:2009.11392, eq. 2.1 and Algorithm 2)
 * approximates a dense m x n matrix A by
 *
 *     A_hat = (AX) (Y^T A X)^+_eps (Y^T A),   X: n x r,  Y: m x (r+l),
 *
 * evaluated in the stable order of eq. 5.1: C = Y^T A X = QR (Householder),
 * F = (AX) R^{-1} by triangular solve, G = Q^T (Y^T A), A_hat = F G.  The
 * stabilised form (SGN, eq. 2.2, Section 5.1.1) truncates R where its diagonal
 * falls to eps and re-factors R_1^T = Q_2 R_2, giving F = (AX) Q_2 R_2^{-T}.
 *
 * Conventions shared by every call
 *   - Matrices are row-major device arrays described by gn_mat: element (i, j)
 *     is at data + i*ld + j.  All pointers in a gn_mat are DEVICE pointers
 *     unless a call says otherwise.  The caller allocates and owns every
 *     buffer; the library never frees caller memory.
 *   - Calls are asynchronous on the handle's CUDA stream.  Argument, shape and
 *     dtype errors are detected on the host and returned before anything is
 *     enqueued.  Device-side failures (a bounded wait that expired, a
 *     non-finite core) are latched in a device status word that
 *     gn_sync_status() returns.
 *   - Scratch memory is a caller-provided device buffer (ws, ws_bytes) sized by
 *     gn_workspace_size(); a call given too small a buffer returns
 *     GN_ERR_WORKSPACE.  Calls that share one workspace must be ordered on one
 *     stream.
 *   - There is no CPU fallback: every step runs in this library's CUDA kernels
 *     (sm_103a).  A missing device or a CUDA error gives GN_ERR_CUDA.
 */
#ifndef GN_H
#define GN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GN_OK = 0,
    GN_ERR_INVALID_ARG = 1,   /* null pointer, bad enum, bad leading dimension */
    GN_ERR_SHAPE = 2,         /* inconsistent sizes, or r, l outside 1 <= r <= min(m,n), l >= 1 */
    GN_ERR_DTYPE = 3,         /* dtype combination not supported by the call */
    GN_ERR_WORKSPACE = 4,     /* ws_bytes below gn_workspace_size() */
    GN_ERR_CUDA = 5,          /* a CUDA runtime / driver call failed */
    GN_ERR_NONFINITE = 6,     /* a non-finite value reached the core */
    GN_ERR_TIMEOUT = 7,       /* a bounded device-side wait expired */
    GN_ERR_UNSUPPORTED = 8,   /* valid request the library does not implement */
    GN_ERR_ALIGNMENT = 9      /* operand address / leading dimension breaks a TMA rule */
} gn_status;

typedef enum {
    GN_F64 = 0,     /* double */
    GN_F32 = 1,     /* float */
    GN_BF16 = 2,    /* bfloat16 (2 bytes) */
    GN_BF16X2 = 3,  /* split bfloat16: value = data + lo, both bf16, same layout */
    GN_E4M3 = 4     /* FP8 e4m3 (1 byte) with one power-of-two scale per 128 x 128
                       tile: value = e4m3(data) * 2^(scale byte - 127) (gn_mat.scale) */
} gn_dtype;

typedef enum {
    GN_MODE_PLAIN = 0,   /* plain GN (eq. 2.1 via eq. 5.1): k = r, F = (AX) R^{-1} */
    GN_MODE_SGN = 1,     /* stabilised GN (eq. 2.2, Section 5.1.1): truncate at eps */
    GN_MODE_AUTO = 2,    /* Section 5.1.2: plain unless est||R^{-1}||_2 * eps >= 100 */
    /* Flag OR'd into the mode: eps is relative to ||C||_2 (estimated by 6 power
     * iterations on R from the all-ones vector), so eps = 10u reproduces the
     * paper's eps = 10u for ||A|| = 1 and O(1) sketches (Section 4.1). */
    GN_EPS_RELATIVE = 0x100,
    /* Flag OR'd into the mode of gn_core (SGN / AUTO): return without waiting
     * for k; the host fields arrive with gn_core_finish (see there). */
    GN_CORE_DEFER = 0x200,
    /* Flag OR'd into the mode of gn_core: core->C already holds C = (Y^T A) X
     * (FP64, (r+l) x r, ld r; for example from gn_countsketch_apply when X is a
     * CountSketch), so gn_core does not form it from YtA and X. */
    GN_CORE_C_GIVEN = 0x400
} gn_mode;

typedef struct {
    void* data;      /* device pointer, row-major */
    void* lo;        /* GN_BF16X2 only: low-order bf16 part (same rows, cols, ld) */
    int64_t rows;
    int64_t cols;
    int64_t ld;      /* leading dimension in elements, >= cols */
    int32_t dtype;   /* gn_dtype */
    /* GN_E4M3 only (NULL / 0 otherwise):
     *   scale : device, ceil(rows/128) x ceil(cols/128) bytes, row-major over
     *           tiles; byte = e + 127 (UE8M0) for the tile's scale 2^e.
     *   data_t: device, the transpose (cols x rows, e4m3, leading dimension
     *           ld_t) under the same scales (its tile (j, i) is tile (i, j)).
     * The tensor cores read every e4m3 operand K-major, so the sketch uses
     * A.data and A.data_t, X.data_t (r x n) and Y.data_t ((r+l) x m). */
    uint8_t* scale;
    void* data_t;
    int64_t ld_t;
} gn_mat;

/* The small core produced by gn_core().  Q, R, Q2, R2, C are caller-allocated
 * DEVICE arrays in FP64; r, l, k, sgn and rinv_est are host fields.
 *   Q   : (r+l) x r, ld = r.  Thin Q of C = Y^T A X; its first k columns are Q_1.
 *   R   : r x r, ld = r.  Upper triangular, diag(R) >= 0.
 *   Q2  : r x r, ld = r.  Q of R_1^T (only the first k columns used; SGN, k < r).
 *   R2  : r x r, ld = r.  R of R_1^T (leading k x k block used; SGN, k < r).
 *   C   : (r+l) x r, ld = r.  The core matrix itself (kept for diagnostics).
 * After gn_core() returns, the host fields hold: k (truncation rank, = r for
 * plain GN), sgn (1 when the truncated branch was taken), rinv_est (the
 * power-method estimate of ||R^{-1}||_2; computed in SGN and AUTO modes,
 * 0 in PLAIN mode), c_norm_est and eps_abs. */
typedef struct {
    double* Q;
    double* R;
    double* Q2;
    double* R2;
    double* C;
    int64_t r;
    int64_t l;
    int64_t k;
    int32_t sgn;
    double rinv_est;
    double c_norm_est;   /* est ||C||_2 (GN_EPS_RELATIVE only, else 0) */
    double eps_abs;      /* absolute truncation threshold that was used */
} gn_core_t;

typedef struct gn_handle_s* gn_handle;

/* ------------------------------------------------------------------ handle */

/* Create a handle bound to the current CUDA device and to `stream` (a
 * cudaStream_t; NULL = legacy default stream).  Allocates one 64-byte device
 * status word.  Returns GN_ERR_CUDA when no device is usable. */
gn_status gn_create(gn_handle* out, void* stream);
gn_status gn_destroy(gn_handle h);
gn_status gn_set_stream(gn_handle h, void* stream);

/* Synchronise the handle's stream, then return (and clear) the latched device
 * status: GN_OK, GN_ERR_TIMEOUT or GN_ERR_NONFINITE, or GN_ERR_CUDA if the
 * stream reported an error. */
gn_status gn_sync_status(gn_handle h);

/* Device-side wait limit in nanoseconds for the pipelined kernels' mbarrier
 * waits (default 2e9).  A wait that exceeds it latches GN_ERR_TIMEOUT, the
 * kernel drains its in-flight copies, frees its tensor memory and returns. */
gn_status gn_set_wait_limit(gn_handle h, uint64_t ns);

/* Test hook for the timeout path above (on = 1 / 0).  While on, the epilogue
 * warps of every tensor-core sketch launch on this handle first wait on an
 * mbarrier that nothing ever completes; that bounded wait runs out after the
 * wait limit, latches GN_ERR_TIMEOUT and stops the launch, whose other roles
 * then drain their copies and MMAs, free tensor memory and return.  The
 * launch's outputs are then incomplete.  Nothing faults or hangs; the handle
 * stays usable once the hook is off.  Off by default. */
gn_status gn_set_stall_test(gn_handle h, int32_t on);

/* Precision of the factor G = Q_1^T (Y^T A) in gn_factors / gn_approx when
 * Y^T A is GN_F32 (the tensor-core sketches).  0 (default): on the tensor
 * cores from three BF16 slices of each factor with FP32 accumulation, i.e. at
 * the precision of an FP32-accumulated Y^T A; 1: an FP64 product, for callers
 * whose sketch reaches beyond FP32 accumulation error (split BF16 aiming at
 * the FP64 path's error).  The triangular solve for F is FP64 either way
 * (eq. 5.1: it carries the conditioning of R). */
gn_status gn_set_fp64_g(gn_handle h, int32_t fp64_g);

/* FP64-level accumulation for callers that need the FP64 path's error from
 * FP32 sketches (split BF16 A): part_k = 0 (default) off; part_k >= 4096 (a
 * multiple of 64) on.  When on: (1) gn_sketch on GN_BF16X2 operands runs the K
 * range of each product as parts of about part_k elements, each accumulated
 * in FP32 in tensor memory, stored, and summed in FP64 (the tensor cores'
 * FP32 accumulation over the full K = m or n is what limits split BF16
 * otherwise); the parts live in the caller's workspace, which
 * gn_workspace_size(..., GN_BF16X2) sizes for part_k = 4096;
 * (2) gn_core forms C = (Y^T A) X from GN_F32 Y^T A and GN_BF16 X by exact
 * digit slicing (FP64 accuracy, as gn_dgemm_tc) instead of FP32-accumulated
 * BF16 slices; (3) gn_factors forms G in FP64 (as gn_set_fp64_g(h, 1)).
 * GN_ERR_INVALID_ARG for other part_k.  The paper fixes no working precision
 * for the sketches; this is the library's. */
gn_status gn_set_fp64_accum(gn_handle h, int64_t part_k);

/* Where the large FP64 products run for GN_F32 sketches (the tensor-core
 * path): in gn_core, the QR's trailing updates (for r >= 512 the
 * factorization runs in 256-column blocks and each block's reflectors update
 * the columns to its right as two products after U = V T; below that, the columns beyond
 * the next two panels of the look-ahead) and the formation of the thin Q; in
 * gn_factors / gn_approx, the outer-block updates of the triangular solve
 * F R = AX (eq. 5.1) and, after a truncation, AX Q_2; in gn_apply, the products
 * with AX and Y^T A.  1 (default): on the BF16 tensor cores by exact digit
 * slicing (gn_dgemm_tc; FP64-level accuracy, about 1e-13 of |A||B| per
 * element); 0: on the FP64 units.  The panels, the small diagonal-block solves
 * and the detector stay in FP64 either way; FP64 sketches always use the FP64
 * units. */
gn_status gn_set_fp64_tc(gn_handle h, int32_t on);

/* C = alpha op(A) op(B) + beta C, FP64 (A may be FP32), computed on the BF16
 * tensor cores by exact digit slicing (the error-free splitting of Ozaki,
 * Ogita, Oishi and Rump, 2012).  Row-major; op(A) is M x K (ta = 0: A[i*lda +
 * k]; ta = 1: A[k*lda + i]), op(B) is K x N (tb = 0: B[k*ldb + j]; tb = 1:
 * B[j*ldb + k]), C is M x N with leading dimension ldc.  Every row of op(A)
 * and column of op(B) is scaled by a power of two and cut into signed 7-bit
 * digits held exactly in BF16 (7 digits per operand); the slice
 * products of each order are summed in FP32 accumulators, exactly for the
 * four leading orders, in passes of at most 1024 of K, and combined in FP64.
 * Error per element about 2^-46 K max_k |op(A)_ik| max_k |op(B)_kj|.
 * Device pointers; ws (device, 256-byte aligned, >= gn_dgemm_tc_workspace_size)
 * is scratch owned by the caller.  GN_ERR_INVALID_ARG for K < 1 or null
 * pointers, GN_ERR_SHAPE for leading dimensions shorter than a row,
 * GN_ERR_ALIGNMENT for an unaligned ws, GN_ERR_WORKSPACE if ws is short.
 * Asynchronous on the handle's stream. */
gn_status gn_dgemm_tc_workspace_size(int64_t M, int64_t N, int64_t K, int32_t a_f32, size_t* bytes);
gn_status gn_dgemm_tc(gn_handle h, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int32_t a_f32,
                      int64_t lda, int32_t ta, const double* B, int64_t ldb, int32_t tb, double beta, double* C,
                      int64_t ldc, void* ws, size_t ws_bytes);

const char* gn_status_string(gn_status s);

/* Number of SMs of the handle's device (the persistent grids use it). */
int gn_device_sm_count(gn_handle h);

/* Total number of CUDA kernels this library has launched in the process
 * (all handles).  A diagnostic counter: differences around a region count the
 * library's launches inside it. */
uint64_t gn_kernel_launches(void);

/* ----------------------------------------------------------------- sizing */

/* Scratch bytes needed by gn_sketch/gn_core/gn_factors/gn_approx/gn_hmt for
 * an m x n problem with sketch sizes r, l whose sketch operands have dtype
 * `op_dtype` (GN_F64 for the plain FP64 path; GN_BF16 / GN_BF16X2 for the
 * tensor-core path).  One buffer of this size serves every call on the shape. */
gn_status gn_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l,
                            int32_t op_dtype, size_t* bytes);

/* ------------------------------------------------------ Algorithm 2, step 1-2 */

/* Operand preparation for the tensor-core path (mixed precision).
 * src: GN_F64 or GN_F32 matrix; dst: same rows/cols, dtype GN_BF16 (round to
 * nearest even via FP32) or GN_BF16X2 (dst.data = bf16(x32), dst.lo =
 * bf16(x32 - hi), x32 = fp32(x)).  dst.ld must be a multiple of 8 and the
 * data (and lo) pointers 16-byte aligned, the layout TMA needs.
 * dst GN_E4M3: per 128 x 128 tile, e = the smallest integer with
 * max|x32| <= 448 * 2^e (0 for a zero tile, clamped to [-127, 127]), and each
 * element becomes e4m3(x32 * 2^-e), rounded to nearest even, saturating.
 * Writes dst.scale (required) and dst.data and / or dst.data_t (either may be
 * NULL); ld and ld_t multiples of 16, pointers 16-byte aligned.  The paper
 * fixes no precision for the sketches (any well-conditioned O(1) sketch
 * works, Section 4); the per-tile scaling is this library's. */
gn_status gn_quantize(gn_handle h, const gn_mat* src, gn_mat* dst);

/* The two sketches of Algorithm 2, step 2: AX (m x r) and Y^T A ((r+l) x n).
 *   A: m x n; X: n x r; Y: m x (r+l) (Y is passed untransposed).
 *   GN_F64 operands: AX, YtA are GN_F64; computed with FP64 FMA.
 *   GN_BF16 / GN_BF16X2 A with GN_BF16 X, Y: one launch of the tcgen05
 *     tensor-core kernel, FP32 accumulation; AX, YtA are GN_F32.  Operand
 *     ld must be a multiple of 8, bases 16-byte aligned (GN_ERR_ALIGNMENT).
 *   GN_E4M3 A, X, Y (with data_t and scale as described at gn_mat): block-
 *     scaled e4m3 tensor-core MMAs (the tile scales as UE8M0 scale factors),
 *     FP32 accumulation; AX, YtA are GN_F32; ld / ld_t multiples of 16.
 * Outputs are overwritten (no accumulation into them). */
gn_status gn_sketch(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y,
                    gn_mat* AX, gn_mat* YtA, void* ws, size_t ws_bytes);

/* The core of Algorithm 2 step 2 and Section 5.1: C = (Y^T A) X, Householder
 * C = QR with diag(R) >= 0, then per `mode` the eps-truncation and the
 * second QR of Section 5.1.1, and (SGN/AUTO) the Section 5.1.2 estimate of
 * ||R^{-1}||_2 by 6 power iterations from the all-ones vector.
 *   YtA: (r+l) x n, GN_F64 or GN_F32; X: n x r, GN_F64 or GN_BF16.
 *   GN_F64 x GN_F64: C in FP64.  GN_F32 x GN_BF16: C from three bf16 slices
 *   of Y^T A on the tensor cores (FP32 accumulate per slice, slices summed in
 *   FP64).
 *   eps >= 0 is an absolute threshold on |R_ii| (the caller scales it).
 * In SGN / AUTO mode the host waits once, for the diagnostics alone (k sizes
 * the second QR and the factors), while the formation of Q continues on the
 * device; PLAIN mode does not wait.  A NaN or infinity in R latches
 * GN_ERR_NONFINITE in the device status word, and in SGN / AUTO mode a NaN
 * estimate also returns GN_ERR_NONFINITE.
 * With GN_CORE_DEFER in `mode` (SGN / AUTO) the call does not wait at all: it
 * returns with core->k = core->sgn = -1 and the handle holds the pending core
 * until gn_core_finish.  The caller may meanwhile enqueue other work (for
 * example the next approximation's sketch on another handle), but must not
 * reuse ws, the core's buffers or this handle's gn_core before finishing. */
gn_status gn_core(gn_handle h, const gn_mat* YtA, const gn_mat* X, double eps, int32_t mode,
                  gn_core_t* core, void* ws, size_t ws_bytes);

/* Completes the core that gn_core left pending on this handle (GN_CORE_DEFER):
 * waits for its diagnostics (not for the rest of the handle's stream), fills
 * k, sgn, rinv_est, c_norm_est and eps_abs, and enqueues the second QR of
 * Section 5.1.1 when the truncated branch is taken.  `core` must be the
 * descriptor given to that gn_core (same R buffer): GN_ERR_INVALID_ARG
 * otherwise; GN_OK at once when nothing is pending and core->k >= 1.  Returns
 * GN_ERR_NONFINITE as gn_core does. */
gn_status gn_core_finish(gn_handle h, gn_core_t* core);

/* ------------------------------------------------------------- Algorithm 2, step 3 */

/* F = (AX) R^{-1} (k = r) or (AX) Q_2 R_2^{-T} (k < r), by blocked triangular
 * solve in FP64, and G = Q_1^T (Y^T A) in FP64 (eq. 5.1; never forms the core
 * pseudoinverse).  AX: m x r and YtA: (r+l) x n in GN_F64 or GN_F32.
 * F: m x k, G: k x n, both GN_F64 (only the first core->k columns / rows are
 * written; F and G may be allocated r wide / r tall). */
gn_status gn_factors(gn_handle h, const gn_mat* AX, const gn_mat* YtA, const gn_core_t* core,
                     gn_mat* F, gn_mat* G, void* ws, size_t ws_bytes);

/* Use of the approximant without forming it (the text after Algorithm 2):
 *   side 0: out (m x kw) = Ahat W   = AX (R^{-1} (Q_1^T (Y^T A W)))      W: n x kw
 *   side 1: out (kw x n) = W Ahat   = (((W AX) R^{-1}) Q_1^T) Y^T A      W: kw x m
 * in the order given there (O((m + n) r kw) work, no m x n matrix); after a
 * truncation (core->sgn, k < r) the core pseudoinverse Q_2 R_2^{-T} Q_1^T
 * (Section 5.1.1) takes the place of R^{-1} Q^T.  AX and Y^T A as gn_sketch
 * wrote them (GN_F64 or GN_F32), core from gn_core; W and out GN_F64,
 * row-major, device.  FP64 products and triangular solves; with GN_F32
 * sketches the products whose size grows with m or n run to FP64 accuracy on
 * the tensor cores by digit slicing (as gn_dgemm_tc) unless gn_set_fp64_tc(h, 0)
 * keeps them on the FP64 units.  ws (device) of at
 * least gn_apply_workspace_size bytes.  GN_ERR_SHAPE / GN_ERR_DTYPE on
 * mismatched operands; asynchronous on the handle's stream. */
gn_status gn_apply_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l, int64_t kw, int32_t side,
                                  size_t* bytes);
gn_status gn_apply(gn_handle h, const gn_mat* AX, const gn_mat* YtA, const gn_core_t* core, const gn_mat* W,
                   gn_mat* out, int32_t side, void* ws, size_t ws_bytes);

/* Streaming update A <- A + E (Section 6): AX += E X and Y^T A += Y^T E, the
 * sketches of E formed exactly as gn_sketch forms those of A (E given the same
 * way: GN_F64, GN_BF16, GN_BF16X2 or GN_E4M3, with the same X, Y) into scratch
 * and added elementwise into AX and YtA (as gn_sketch wrote them).  The core
 * of the updated sketches is then gn_core's.  ws (device) of at least
 * gn_update_workspace_size(m, n, r, l, dtype of E) bytes, which needs only
 * m, n, r >= 1 and l >= 0 (the same sizing serves gn_append_rows /
 * gn_append_cols for a block B of any size, one row or column included);
 * asynchronous on the handle's stream. */
gn_status gn_update_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l, int32_t op_dtype, size_t* bytes);
gn_status gn_update(gn_handle h, const gn_mat* E, const gn_mat* X, const gn_mat* Y, gn_mat* AX, gn_mat* YtA,
                    void* ws, size_t ws_bytes);

/* Resampling r -> r + dr (Section 6): AXn (m x (r + dr)) = [AX, A Xd] and
 * YtAn ((r + l + dr + dl) x n) = [Y^T A; Yd^T A] from the old sketches (copied)
 * and the sketch of A by the new blocks Xd (n x dr), Yd (m x (dr + dl)) alone,
 * with dr >= 0, dl >= 0 and dr + dl >= 1: dl = 0 raises r keeping l, dr = 0
 * raises l alone (Xd then has no columns and neither it nor AXn's new part is
 * read).  AX, YtA as gn_sketch wrote them, AXn / YtAn of the same dtype, A,
 * Xd, Yd as gn_sketch takes them.  The core of the new state is gn_core's on
 * YtAn and [X, Xd].  ws (device, not NULL) of at least
 * gn_resample_workspace_size(m, n, dr, dl, dtype of A) bytes; GN_ERR_SHAPE for
 * dr < 0, dl < 0 or dr + dl = 0. */
gn_status gn_resample_workspace_size(int64_t m, int64_t n, int64_t dr, int64_t dl, int32_t op_dtype,
                                     size_t* bytes);
gn_status gn_resample(gn_handle h, const gn_mat* A, const gn_mat* Xd, const gn_mat* Yd, const gn_mat* AX,
                      const gn_mat* YtA, gn_mat* AXn, gn_mat* YtAn, void* ws, size_t ws_bytes);

/* Appended data (Section 6).  Rows [A; B], B (mb x n) with a new sketch block
 * Yb (mb x (r + l)): AXn ((m + mb) x r) = [AX; B X], Y^T A += Yb^T B (in place).
 * Columns [A, B], B (m x nb) with a new sketch block Xb (nb x r): AX += B Xb
 * (in place), YtAn ((r + l) x (n + nb)) = [Y^T A, Y^T B].  Operands as for
 * gn_update; ws: gn_update_workspace_size for B's shape. */
gn_status gn_append_rows(gn_handle h, const gn_mat* B, const gn_mat* X, const gn_mat* Yb, const gn_mat* AX,
                         gn_mat* YtA, gn_mat* AXn, void* ws, size_t ws_bytes);
gn_status gn_append_cols(gn_handle h, const gn_mat* B, const gn_mat* Xb, const gn_mat* Y, gn_mat* AX,
                         const gn_mat* YtA, gn_mat* YtAn, void* ws, size_t ws_bytes);

/* ------------------------------------------------------- structured sketches */

/* The subsampled DCT sketch matrix of Section 7's experiments (Section 2.5's
 * fast sketches): X = D C^T S (n x r), D = diag(signs) (device, n doubles, +-1),
 * C the orthonormal DCT-II matrix C[k, i] = a_k cos(pi (2 i + 1) k / (2 n))
 * (a_0 = sqrt(1/n), a_k = sqrt(2/n)), S the columns cols[0..r-1] of the
 * identity (device, r int64 in [0, n), distinct).  X has orthonormal columns;
 * the sqrt(n/r) scale is left out (GN is invariant under X -> X c).  Written
 * into X (n x r, GN_F64, GN_F32 or GN_BF16 rounded through FP32 like
 * gn_quantize; BF16 ld a multiple of 8, 16-byte base), so the sketches of
 * A with X (and with Y = a DCT sketch of m) then run through gn_sketch.  The
 * same call makes Y (m x (r + l)) from its own draws.  GN_ERR_SHAPE unless
 * 1 <= r <= n <= 2^31 and X is n x r. */
gn_status gn_dct_sketch(gn_handle h, int64_t n, int64_t r, const double* signs, const int64_t* cols, gn_mat* X);

/* A sparse m x n matrix in CSR form (device arrays): row_ptr (m + 1 int64,
 * row_ptr[0] = 0, row_ptr[m] = nnz, non-decreasing), col_idx (nnz int32 in
 * [0, n)), vals (nnz entries of `dtype`, GN_F64 or GN_F32). */
typedef struct {
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const void* vals;
    int64_t rows, cols, nnz;
    int32_t dtype;
} gn_csr;

/* The sketches of a sparse A with CountSketch sketches (Section 2.5's
 * input-sparsity route; Section 7's sparse experiment): X (n x r) has one
 * entry per row, X[j, bx[j]] = sx[j], and Y (m x (r + l)) likewise with by,
 * sy (device arrays: bx n int64 in [0, r), sx n doubles, by m int64 in
 * [0, r + l), sy m doubles).  AX (m x r) and YtA ((r + l) x n), of A's dtype,
 * are overwritten in O(nnz) work: every nonzero a_ij adds sx[j] a_ij to
 * AX[i, bx[j]] and sy[i] a_ij to YtA[by[i], j] (device atomic adds; the
 * order of the additions is not fixed).  r and r + l are AX->cols and
 * YtA->rows; either output may be NULL to skip it.  A column index or bucket
 * outside its range skips that nonzero and latches GN_ERR_INVALID_ARG in the
 * device status word (gn_sync_status).  The core of the sketch state is then
 * gn_core's, with X given densely by gn_countsketch_matrix. */
gn_status gn_sketch_csr_countsketch(gn_handle h, const gn_csr* A, const int64_t* bx, const double* sx,
                                    const int64_t* by, const double* sy, gn_mat* AX, gn_mat* YtA);

/* out (rows x r, GN_F64) = B X for a dense B (rows x n, GN_F64 or GN_F32) and
 * the CountSketch X of the draws bx, sx (as above): column c of out is the
 * signed sum of the columns j of B with bx[j] = c, in O(rows n) work (device
 * FP64 atomic adds; the order of the additions is not fixed).  With B = Y^T A
 * this is the core C = (Y^T A) X for gn_core's GN_CORE_C_GIVEN.  A bucket
 * outside [0, r) latches GN_ERR_INVALID_ARG and skips that column. */
gn_status gn_countsketch_apply(gn_handle h, const gn_mat* B, const int64_t* bx, const double* sx, gn_mat* out);

/* The dense CountSketch matrix (n x r, GN_F64 or GN_F32): X[i, buckets[i]] =
 * signs[i], zero elsewhere (device draws as for gn_sketch_csr_countsketch). */
gn_status gn_countsketch_matrix(gn_handle h, int64_t n, int64_t r, const int64_t* buckets, const double* signs,
                                gn_mat* X);

/* ------------------------------------------ Section 5.1.1's perturbed cores */

/* The alternatives of Section 5.1.1 to truncating R, and SGN with the SVD
 * epsilon-pseudoinverse (eq. 2.2), from a sketch state:
 *   GN_VARIANT_SVD_TRUNCATE: C = U S V^T, keep s_i > eps:
 *                            F = AX V_k S_k^{-1}, G = U_k^T (Y^T A)
 *   GN_VARIANT_SVD_RAISE   : s_i -> max(s_i, eps): F = AX V S~^{-1}, G = U^T (Y^T A)
 *   GN_VARIANT_RRQR_RAISE  : column-pivoted Householder C P = Q R (the column of
 *                            largest remaining norm first), |R_ii| -> max(|R_ii|, eps)
 *                            with the sign kept: F = (AX P) R~^{-1}, G = Q^T (Y^T A)
 *   GN_VARIANT_DIAG_RAISE  : unpivoted C = Q R with |R_ii| raised the same way:
 *                            F = AX R~^{-1}, G = Q^T (Y^T A)
 * eps is absolute (the caller scales it); the raising variants need eps > 0.
 * C = (Y^T A) X is formed in FP64; every product and solve is FP64.  AX (m x r)
 * and YtA ((r+l) x n): both GN_F64 or both GN_F32; X (n x r): GN_F64 or GN_BF16;
 * F (m x >= r) and G (>= r x n) GN_F64, their first k columns / rows written.
 * *k_out (host) receives k (r except for SVD_TRUNCATE); sv (device, r doubles,
 * optional) the singular values by decreasing size (SVD variants) or diag(R)
 * before raising (QR variants).  The SVD and pivoted variants factor C in one
 * CTA's shared memory (one-sided Jacobi rotations; pivoted Householder) and
 * need r <= 128 and r + l <= 192 (GN_ERR_UNSUPPORTED otherwise); DIAG_RAISE
 * takes any r.  Blocks the host once for k (SVD and pivoted variants).
 * GN_ERR_NONFINITE when k = 0.  ws: gn_variant_workspace_size bytes. */
typedef enum {
    GN_VARIANT_SVD_TRUNCATE = 0,
    GN_VARIANT_SVD_RAISE = 1,
    GN_VARIANT_RRQR_RAISE = 2,
    GN_VARIANT_DIAG_RAISE = 3
} gn_variant;
gn_status gn_variant_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l, size_t* bytes);
gn_status gn_factors_variant(gn_handle h, const gn_mat* AX, const gn_mat* YtA, const gn_mat* X, double eps,
                             int32_t variant, gn_mat* F, gn_mat* G, int64_t* k_out, double* sv, void* ws,
                             size_t ws_bytes);

/* Sketch + core + factors in one call (Algorithm 2).  AX, YtA are outputs
 * (GN_F64 for FP64 operands, GN_F32 for the tensor-core path). */
gn_status gn_approx(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y,
                    double eps, int32_t mode, gn_mat* AX, gn_mat* YtA, gn_core_t* core,
                    gn_mat* F, gn_mat* G, void* ws, size_t ws_bytes);

/* ||A - F G||_F^2 accumulated in FP64 without storing F G (the accuracy measure
 * of Section 7.1).  A: m x n GN_F64, GN_F32, GN_BF16 or GN_BF16X2 (data+lo);
 * F: m x k GN_F64; G: k x n GN_F64.  The result is written to the DEVICE
 * double *out (overwritten). */
gn_status gn_error_fro2(gn_handle h, const gn_mat* A, const gn_mat* F, const gn_mat* G,
                        double* out, void* ws, size_t ws_bytes);

/* Allocation-free ||A - F G||_F^2, for callers that cannot allocate device
 * memory: for example code that runs inside a host application whose memory
 * manager owns the whole device and refuses further cudaMalloc calls, or a
 * latency-critical loop that must not allocate.  The paper has no counterpart;
 * this is a convenience of the library.
 * Same arguments, arithmetic and result as gn_error_fro2, but no workspace: the
 * per-tile partial sums live in one fixed array in device memory that every
 * GPU loading the library holds until the process exits (128 KB).  Limit:
 * ceil(m/64) * ceil(n/64) <= 16384 tiles (about 67 million elements of A, e.g.
 * 8192 x 8192); larger sizes return GN_ERR_SHAPE before anything runs.  No
 * device memory is allocated by this call.  The first call on a device looks
 * up the array's device address (once per device, with that device made
 * current); make that first call before any stream capture.  All calls share
 * the one array and each overwrites every slot it reads, so its previous
 * contents never matter -- but calls whose kernels overlap on the GPU (for
 * example on two streams at once) race on the array and give wrong results;
 * order them on one stream. */
gn_status gn_error_fro2_noalloc(gn_handle h, const gn_mat* A, const gn_mat* F, const gn_mat* G,
                                double* out);

/* ------------------------------------------------ adjoint of A -> A_hat (plain GN) */

/* Scratch bytes for gn_backward / gn_forward_dense on an m x n input with
 * sketch sizes r, l in `dtype` (GN_F64 or GN_F32). */
gn_status gn_backward_workspace_size(int64_t m, int64_t n, int64_t r, int64_t l, int32_t dtype,
                                     size_t* bytes);

/* Gradient of L(A) = <Gup, A_hat(A)> for plain GN (eq. 2.1 evaluated as in
 * eq. 5.1) with X, Y held fixed, for a core Y^T A X of full column rank:
 *   dA = (S1 Q R^{-T} + Y K) X^T + Y (Q S2),   S1 = Gup (Y^T A)^T,
 *   F = (AX) R^{-1},  S2 = F^T Gup,  W = F^T S1,
 *   K = (I - Q Q^T) W^T R^{-T} - Q (W Q) R^{-T},
 * derived from d(C^+) = -C^+ dC C^+ + (C^T C)^{-1} dC^T (I - C C^+) (the
 * paper does not differentiate GN).  The core's pseudoinverse is never formed.
 * A, X, Y, Gup, dA share one dtype: GN_F64 (every step in FP64) or GN_F32
 * (the m x n contractions in FP32, the r-sized algebra in FP64).  A: m x n,
 * X: n x r, Y: m x (r+l), Gup, dA: m x n (dA overwritten).  The sketches,
 * C = QR and F are formed from A in ws (the "front") and left there for
 * gn_backward_saved.  FP32: data 16-byte aligned, ld a multiple of 4 (dA
 * exempt from the ld rule); GN_ERR_ALIGNMENT otherwise. */
gn_status gn_backward(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y,
                      const gn_mat* Gup, gn_mat* dA, void* ws, size_t ws_bytes);

/* The dense approximant A_hat = F G (m x n) of plain GN in the dtype of A
 * (GN_F64 or GN_F32, same precision split as gn_backward); the forward value
 * of the differentiable map whose adjoint gn_backward computes.  Forms the
 * same front in ws as gn_backward and leaves it there. */
gn_status gn_forward_dense(gn_handle h, const gn_mat* A, const gn_mat* X, const gn_mat* Y,
                           gn_mat* Ahat, void* ws, size_t ws_bytes);

/* gn_backward from the front that the handle's last gn_forward_dense or
 * gn_backward call left in ws (what an autograd forward saves for its
 * backward): the same dA, without the sketches, the core's QR and F.  A is not
 * read.  X, Y must be the matrices of that call (same pointers and leading
 * dimensions), Gup and dA m x n in its dtype, ws and ws_bytes the same, and
 * ws untouched since; the handle keeps one such record (a later
 * gn_forward_dense or gn_backward replaces it).  GN_ERR_INVALID_ARG when the
 * record does not match (checked on the host); may be called again with
 * another Gup.  Asynchronous on the handle's stream. */
gn_status gn_backward_saved(gn_handle h, const gn_mat* X, const gn_mat* Y, const gn_mat* Gup,
                            gn_mat* dA, void* ws, size_t ws_bytes);

/* ---------------------------------------------------------------- batched */

/* One problem of a batch (uneven m, n, r, l allowed).  Inputs GN_BF16 (ld a
 * multiple of 8, 16-byte aligned); outputs AX, YtA GN_F32; core buffers FP64
 * device arrays: Q (r+l) x r, R, Q2, R2 r x r (all ld r); k: device int32 that
 * receives the truncation rank (r unless the truncated branch was taken).
 * Limits of the shared-memory core: r <= 128 and r + l <= 192. */
typedef struct {
    gn_mat A, X, Y;
    gn_mat AX, YtA;
    double* Q;
    double* R;
    double* Q2;
    double* R2;
    int32_t* k;
} gn_problem;

/* Workspace bytes for a batch (tables, tensor maps, slices of Y^T A). */
gn_status gn_batched_workspace_size(int32_t count, const gn_problem* probs, size_t* bytes);

/* Build and upload the batch's descriptors (GEMM tiles, TMA tensor maps,
 * per-problem scratch layout) into `ws`.  Synchronous; call once per batch
 * layout (pointers and shapes), before any capture of gn_batched_run. */
gn_status gn_batched_prepare(gn_handle h, int32_t count, const gn_problem* probs, void* ws,
                             size_t ws_bytes);

/* Tile policy of the batch's tensor-core launches, used by the next
 * gn_batched_prepare (bit field; 0 = the fixed rule):
 *   bits 0-1: N tile of every Y^T A product: 0 -> 128, 1 -> 64, 2 -> 256
 *   bit 2   : N tile 64 for AX when 64 < r (two tiles instead of one)
 *   bit 3   : problems ordered by decreasing sketch work in the tile list
 *   bit 4   : 256-row sketch tiles (two M halves share each B stage)
 * The paper has no batched mode; the policy is this library's. */
#define GN_BATCHED_POLICIES 24
gn_status gn_batched_set_policy(gn_handle h, int32_t policy);

/* Autotuner: for each of the GN_BATCHED_POLICIES policies, prepare the batch
 * and time gn_batched_run (one warm-up, three timed runs, CUDA events on the
 * handle's stream); then prepare it again with the fastest, which stays set
 * on the handle and is written to *best (ms per run to *best_ms if non-null).
 * Synchronous; overwrites the problems' outputs. */
gn_status gn_batched_tune(gn_handle h, int32_t count, const gn_problem* probs, void* ws, size_t ws_bytes,
                          double eps, int32_t mode, int32_t* best, double* best_ms);

/* Algorithm 2 step 2 and the Section 5.1 core for every prepared problem, in
 * four launches on the handle's stream: one grouped tensor-core launch for
 * all sketches AX, Y^T A (BF16, FP32 accumulation), one split of every Y^T A
 * into three BF16 slices, one grouped launch for the slice products of every
 * core C = (Y^T A) X, and one kernel with a CTA per problem (FP64 Householder
 * QR and Q in shared memory, diag(R) >= 0, the Section 5.1.2 detector and
 * Section 5.1.1 truncation per `mode` / `eps` exactly as gn_core, second QR
 * into Q2, R2 when truncated).  No host synchronisation and no allocation;
 * `ws` must be the workspace given to gn_batched_prepare. */
gn_status gn_batched_run(gn_handle h, double eps, int32_t mode, void* ws, size_t ws_bytes);

/* ---------------------------------------------------------------- Algorithm 1 */

/* HMT range finder (Algorithm 1): AX, Householder QR AX = Q R_x, B = Q^T A.
 * All GN_F64: A m x n, X n x r, Q m x r (output), B r x n (output). */
gn_status gn_hmt(gn_handle h, const gn_mat* A, const gn_mat* X, gn_mat* Q, gn_mat* B,
                 void* ws, size_t ws_bytes);

#ifdef __cplusplus
}
#endif
#endif /* GN_H */
