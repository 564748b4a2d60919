/*
 * qrkit.h - C ABI of a GB300 (sm_103a) library that solves the damped least-squares
 * problem of a Levenberg-Marquardt step by structured sparse QR.
 *
 * The operation (arXiv 1802.03773, Eq. 2):   min_p || [J; lambda^(1/2) D] p - [b; 0] ||_2,
 * equivalently the normal equations Eq. 1, (J^T J + lambda D^2) p = J^T b, solved without
 * forming J^T J.  J is given by a structure descriptor plus packed values:
 *   QRKIT_STRUCT_BLOCKS   J = [blkdiag(J_1..J_K) | S]          (Sec. 4.1 block diagonal,
 *                         Sec. 4.2 horizontal concatenation); S absent, dense, or windowed
 *   QRKIT_STRUCT_BANDED   J banded: row i touches w consecutive columns from
 *                         floor(i / rows_per_col) (Sec. 4.4 block banded)
 * The damping rows lambda^(1/2) D are appended by the row interleave of Sec. 4.5 / Sec. 5.2
 * ("Backtrack LM"): P_r [J; lambda^(1/2) D] = Q R, factored once.
 *
 * Conventions for every entry point:
 *   - All value buffers are DEVICE pointers (memory of the context's device), owned by the
 *     caller, on the stream given to qrkit_create; calls are asynchronous on that stream
 *     unless stated.  Index/shape arrays inside qrkit_structure are HOST pointers, read
 *     during qrkit_plan only.
 *   - Value precision follows the context: float for QRKIT_FP32 / QRKIT_FP32_REFINED,
 *     double for QRKIT_FP64.  lambda is always a double.
 *   - Every function returns a qrkit_status; nothing throws across the ABI.  On error a
 *     message is kept per context (qrkit_last_error).  Device-side failures (non-finite
 *     input, zero pivot) are recorded in a device status word, read by qrkit_sync_status.
 *   - Householder convention (Sec. 2): reflector H = I - tau v v^T with v[0] = 1,
 *     beta = -sign(x0) ||x||, tau = (beta - x0) / beta; R may have negative diagonal.
 */
#ifndef QRKIT_H
#define QRKIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QRKIT_OK = 0,
  QRKIT_EINVAL = 1,       /* bad argument or descriptor */
  QRKIT_ENOMEM = 2,       /* device allocation failed */
  QRKIT_ECUDA = 3,        /* a CUDA runtime call failed */
  QRKIT_ESINGULAR = 4,    /* a diagonal entry of R is zero */
  QRKIT_ENONFINITE = 5,   /* NaN/Inf met in the inputs or the factor */
  QRKIT_ETIMEOUT = 6,     /* a bounded device wait expired */
  QRKIT_ENOTCONV = 7,     /* LM stopped without converging */
  QRKIT_EUNSUPPORTED = 8, /* structure or size outside what this build handles */
  QRKIT_ESTATE = 9        /* call order: e.g. solve before factor, factor before plan */
} qrkit_status;

typedef enum {
  QRKIT_FP64 = 0,          /* all arithmetic in double */
  QRKIT_FP32_REFINED = 1,  /* float factors, high-precision residual refinement */
  QRKIT_FP32 = 2           /* float factors, no refinement */
} qrkit_precision;

typedef enum { QRKIT_STRUCT_BLOCKS = 0, QRKIT_STRUCT_BANDED = 1 } qrkit_struct_kind;
typedef enum {
  QRKIT_COUPLED_NONE = 0,   /* J = blkdiag(J_i) */
  QRKIT_COUPLED_DENSE = 1,  /* J = [blkdiag(J_i) | S], S dense (sum n_i) x s, column-major */
  QRKIT_COUPLED_WINDOW = 2  /* block i's rows touch S columns start_i .. start_i + w - 1 */
} qrkit_coupled_kind;

/* Structure descriptor (the paper's compile-time composition, Sec. 3 / Sec. 5.1, as data). */
typedef struct qrkit_structure {
  int32_t kind;                 /* qrkit_struct_kind */
  /* --- QRKIT_STRUCT_BLOCKS --- */
  int64_t num_blocks;           /* K >= 1 */
  const uint8_t* block_rows;    /* host, K entries: n_i (J rows of block i), 1..16 */
  const uint8_t* block_cols;    /* host, K entries: m_i, 1..8; with the damping rows the
                                   augmented block has n_i + m_i <= 16 rows (n_i >= m_i
                                   when lambda = 0) */
  int32_t coupled_kind;         /* qrkit_coupled_kind */
  int64_t shared_cols;          /* s: columns of S (0 for QRKIT_COUPLED_NONE) */
  int32_t window;               /* w for QRKIT_COUPLED_WINDOW */
  const int32_t* window_start;  /* host, K entries, non-decreasing, start_i + w <= s + w - 1 */
  /* --- QRKIT_STRUCT_BANDED --- */
  int64_t rows, cols;           /* one instance: J is (rows_per_col * cols) x cols */
  int32_t rows_per_col;         /* row i starts at column floor(i / rows_per_col) */
  int32_t band_window;          /* w: values per row, 1..16 (entries past the last column
                                   are ignored) */
  const int64_t* instance_cols; /* host, num_blocks entries: a batch of independent banded
                                   instances with these column counts (NULL: one instance
                                   of `cols` columns) */
} qrkit_structure;

typedef struct qrkit_ctx qrkit_ctx;

/* Create a context on `device` (CUDA ordinal) issuing work on `stream` (a cudaStream_t,
 * NULL = legacy default stream).  precision: qrkit_precision.  *out receives the context. */
qrkit_status qrkit_create(qrkit_ctx** out, int device, void* stream, int precision);

/* Release the context, its plan and its device workspace.  NULL is allowed. */
void qrkit_destroy(qrkit_ctx* ctx);

/* Message of the last failed call on ctx ("" if none); valid until the next call. */
const char* qrkit_last_error(const qrkit_ctx* ctx);

/* Static name of a status code. */
const char* qrkit_status_string(int status);

/* Structure plan (Sec. 3 composition, Sec. 4.3 / 4.5 row permutation): validates the
 * descriptor, builds offsets, the P_r interleave of the damping rows, the tile schedule of
 * the persistent kernels, and allocates the device workspace that holds the factor.
 * Host work, once per structure; synchronous.  Replaces any previous plan. */
qrkit_status qrkit_plan(qrkit_ctx* ctx, const qrkit_structure* s);

/* Fused factor + solve for QRKIT_STRUCT_BLOCKS with QRKIT_COUPLED_NONE (Sec. 4.1, Sec. 5.1):
 * for every block the Householder QR of J_i, c_i = Q_i^T b_i, R_i p_i = c_i, then (FP32 refined
 * mode) up to `refine_steps` steps of refinement with an extended-precision residual: each
 * step computes g = J_i^T (b_i - J_i p_i) in compensated float arithmetic and corrects
 * p_i += R_i^{-1} R_i^{-T} g; a block stops as soon as its correction is below 1e-6 of its
 * solution (max norms).  refine_steps is ignored for QRKIT_FP32 and QRKIT_FP64.
 *   J    : packed values, block i column-major n_i x m_i, blocks in order (sum n_i m_i)
 *   b    : sum n_i values, block i's rows contiguous
 *   D    : reserved, pass NULL
 *   lambda : must be 0 on this fused path (damped blocks go through qrkit_factor)
 *   p    : out, sum m_i values
 *   qtb  : out or NULL; sum n_i values: Q_i^T b_i per block
 * The factor (reflectors below the diagonal, R on and above it, tau) stays in the context.
 * One kernel launch; asynchronous on the context's stream. */
qrkit_status qrkit_factor_solve(qrkit_ctx* ctx, const void* J, const void* b, const void* D,
                                double lambda, void* p, void* qtb, int refine_steps);

/* For a QRKIT_STRUCT_BANDED plan, qrkit_factor_solve factors and solves every instance of
 * the batch (Sec. 4.4 block-banded QR, damping rows interleaved per column as in Sec. 4.5 /
 * Sec. 5.2): J holds the instances' rows back to back, row-major with band_window values per
 * row; b one value per row; D (total columns, or NULL for column norms, zero -> 1) as above;
 * lambda >= 0; p one value per column; qtb must be NULL; refine_steps: steps of refinement
 * with a double residual (FP32 refined mode).  Q is not kept. */

/* Composed factorization (Sec. 3 composition; Sec. 4.1 block diagonal, Sec. 4.2 horizontal
 * concatenation, Sec. 4.5 vertical concatenation of the damping rows, Sec. 5.2 Backtrack LM):
 * QR of P_r [J; lambda^(1/2) D] for a QRKIT_STRUCT_BLOCKS plan (any coupled_kind).
 *   J    : block values as for qrkit_factor_solve
 *   S    : coupled values or NULL for QRKIT_COUPLED_NONE.  DENSE: (sum n_i) x s column-major;
 *          WINDOW: per block an n_i x w column-major slab, blocks in order
 *   D    : N = sum m_i + s diagonal values, or NULL for the column norms of J (zero -> 1).
 *          Internally kept in double.
 *   lambda >= 0; the damping rows exist only when lambda > 0.
 * The factor (per-block reflectors and R, R12 = Q_i^T S_i top rows, the factor of the
 * reduced shared block) is kept in the context.  J and S are read again by qrkit_solve when
 * refine_steps > 0: keep them alive and unchanged until then.  Dense S: s <= 64. */
qrkit_status qrkit_factor(qrkit_ctx* ctx, const void* J, const void* S, const void* D, double lambda);

/* qtb = Q^T [b; 0] restricted to its top N entries (Sec. 5.1, matrixQ().transpose() * b),
 * laid out as [c_blocks (sum m_i, column order) ; c_S (s)].  b: sum n_i values. */
qrkit_status qrkit_apply_qt(qrkit_ctx* ctx, const void* b, void* qtb);

/* p = R^{-1} qtb (Sec. 5.1, matrixR().solve): qtb as produced by qrkit_apply_qt; p: N values
 * (block columns then shared columns). */
qrkit_status qrkit_solve_r(qrkit_ctx* ctx, const void* qtb, void* p);

/* p = argmin ||P_r [J; lambda^(1/2) D] p - P_r [b; 0]|| with the stored factor: Q^T b,
 * back-substitution, then `refine_steps` refinement steps (QRKIT_FP32_REFINED: residual
 * g = J^T (b - J p) - lambda D^2 p in double, correction R^{-1} R^{-T} g; ignored for
 * QRKIT_FP32, allowed but not useful for QRKIT_FP64). */
qrkit_status qrkit_solve(qrkit_ctx* ctx, const void* b, void* p, int refine_steps);

/* Size of the device array behind qrkit_block_solve_noalloc (16 MiB per device). */
#define QRKIT_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Block-diagonal factor + solve that allocates no device memory.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc, such as code running
 * under a framework that owns all device memory through its own pool, or a process whose
 * device memory budget is fixed when it starts.
 * It solves the same problem as qrkit_plan + qrkit_factor_solve for QRKIT_STRUCT_BLOCKS /
 * QRKIT_COUPLED_NONE with lambda = 0 and no qtb output, without a context:
 *   device, stream, precision : as for qrkit_create (stream: a cudaStream_t or NULL)
 *   block_rows, block_cols    : HOST arrays of num_blocks shapes (1 <= m_i <= n_i <= 16, m_i <= 8)
 *   J, b, p                   : DEVICE buffers as for qrkit_factor_solve (caller-owned)
 *   refine_steps              : as for qrkit_factor_solve (FP32 refined mode only)
 * All intermediates (shapes, tile schedule, factor, tau, status word) live in one device array
 * of QRKIT_NOALLOC_SCRATCH_BYTES that is part of the library image: every process that loads
 * the library holds it on each device it uses until the process exits.  A problem whose
 * intermediates do not fit (roughly sum n_i m_i above 3.5 million values in FP32, half that
 * in FP64) is rejected with QRKIT_EUNSUPPORTED before anything is launched; bad arguments give
 * QRKIT_EINVAL, a failed CUDA call QRKIT_ECUDA.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  Each call copies the
 * shapes and schedule into the array, clears its status word, launches one kernel on `stream`,
 * then waits for the stream and returns the kernel's status (QRKIT_OK, QRKIT_ESINGULAR, ...).
 * Every call uses the same array and leaves its contents behind: calls whose work overlaps on
 * the GPU (other threads, other streams) race and must be serialized by the caller.  The
 * factor is not kept for later calls. */
qrkit_status qrkit_block_solve_noalloc(int device, void* stream, int precision,
                                       int64_t num_blocks, const uint8_t* block_rows,
                                       const uint8_t* block_cols, const void* J, const void* b,
                                       void* p, int refine_steps);

/* Banded factor of the last qrkit_factor_solve on a QRKIT_STRUCT_BANDED plan (device pointers,
 * any may be NULL): Rw[j * w + t] = R[j, j + t] per global column j, c = top of Q^T [b; 0] per
 * column; res2 (HOST, one double per instance) = squared residual norm.  Synchronous. */
qrkit_status qrkit_get_band_factor(qrkit_ctx* ctx, void* Rw, void* c, double* res2);

/* Copy the stored factor of a block structure to caller buffers (device pointers, either
 * may be NULL): factor values in J's packing (V strictly below the diagonal, R on and above)
 * and tau (sum m_i). */
qrkit_status qrkit_get_factor(qrkit_ctx* ctx, void* factor_out, void* tau_out);

/* Block until the stream is idle and return the device status word (QRKIT_OK if no kernel
 * reported a failure), then clear it. */
qrkit_status qrkit_sync_status(qrkit_ctx* ctx);

/* Number of this library's kernels launched on ctx since creation (for launch accounting). */
int64_t qrkit_launch_count(const qrkit_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* QRKIT_H */
