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
  const int32_t* window_start;  /* host, K entries: first S column of block i's window, inside
                                   its segment (below).  Any order: the rows of the reduced
                                   block are sorted by start on the device (Sec. 4.3 P_r).
                                   Window entries past the end of the segment must be zero. */
  /* --- QRKIT_STRUCT_BANDED --- */
  int64_t rows, cols;           /* one instance: J is (rows_per_col * cols) x cols */
  int32_t rows_per_col;         /* row i starts at column floor(i / rows_per_col) */
  int32_t band_window;          /* w: values per row, 1..16 (entries past the last column
                                   are ignored) */
  const int64_t* instance_cols; /* host, num_blocks entries: a batch of independent banded
                                   instances with these column counts (NULL: one instance
                                   of `cols` columns) */
  /* --- QRKIT_COUPLED_WINDOW, optional: S split into independent segments --- */
  int64_t num_segments;          /* 0 or 1: one segment of all s columns */
  const int64_t* segment_cols;   /* host, num_segments entries >= 1 summing to s: columns of
                                    each segment; a window never crosses a segment boundary,
                                    so each segment's reduced block is a separate banded
                                    matrix, solved in parallel with the others */
  const int64_t* segment_blocks; /* host, num_segments entries summing to K: the blocks are
                                    grouped by segment in order, this many per segment */
  /* --- QRKIT_STRUCT_BANDED: algorithm --- */
  int32_t band_solver;           /* QRKIT_BAND_AUTO, QRKIT_BAND_SWEEP or QRKIT_BAND_PARALLEL */
  /* --- QRKIT_STRUCT_BANDED, optional: explicit row starts (Sec. 4.3 row and column
   *     permutations applied by the caller, e.g. those of qrkit_band_order) --- */
  const int32_t* band_row_start; /* host, one entry per row (instances' rows back to back): the
                                    first column of the row inside its instance, non-decreasing
                                    within an instance; NULL: the implicit floor(i / rows_per_col)
                                    rule (rows_per_col is then ignored) */
  const int64_t* instance_rows;  /* host, num_blocks entries: rows of each instance when
                                    band_row_start is given (NULL for one instance: `rows`) */
} qrkit_structure;

/* Banded QR algorithms (both Sec. 4.4 block-banded Householder QR with the damping rows
 * interleaved):
 *   SWEEP     one warp per instance sweeps the column groups in order, carrying the trailing
 *             triangle; R comes out in natural column order (qrkit_get_band_factor).
 *   PARALLEL  rows compressed per block of 8 columns, then block cyclic reduction over the
 *             blocks (log-depth, all blocks of a level in parallel); R is that of the columns
 *             in nested-dissection order and is not exported.  Needs band_window <= 8.
 *   AUTO      PARALLEL when band_window <= 8, else SWEEP. */
enum { QRKIT_BAND_AUTO = 0, QRKIT_BAND_SWEEP = 1, QRKIT_BAND_PARALLEL = 2 };

typedef struct qrkit_ctx qrkit_ctx;

/* Create a context on `device` (CUDA ordinal) issuing work on `stream` (a cudaStream_t,
 * NULL = legacy default stream).  precision: qrkit_precision.  *out receives the context.
 * (No paper counterpart: the context owns the plan and the device workspace.) */
qrkit_status qrkit_create(qrkit_ctx** out, int device, void* stream, int precision);

/* Release the context, its plan and its device workspace.  NULL is allowed.  (No paper
 * counterpart.) */
void qrkit_destroy(qrkit_ctx* ctx);

/* Message of the last failed call on ctx ("" if none); valid until the next call.  (No paper
 * counterpart.) */
const char* qrkit_last_error(const qrkit_ctx* ctx);

/* Static name of a status code.  (No paper counterpart.) */
const char* qrkit_status_string(int status);

/* Structure plan (Sec. 3 composition, Sec. 4.3 / 4.5 row permutation): validates the
 * descriptor, builds offsets, the P_r interleave of the damping rows, the work lists of the
 * persistent kernels (for uncoupled blocks: shape-uniform warp tasks, blocks sorted by shape
 * inside supertiles of consecutive blocks), and allocates the device workspace that holds
 * the factor.
 * Host work, once per structure; synchronous.  Replaces any previous plan. */
qrkit_status qrkit_plan(qrkit_ctx* ctx, const qrkit_structure* s);

/* Fused factor + solve for QRKIT_STRUCT_BLOCKS with QRKIT_COUPLED_NONE (Sec. 4.1, Sec. 5.1):
 * for every block the Householder QR of J_i, c_i = Q_i^T b_i, R_i p_i = c_i.  In FP32 refined
 * mode each block then bounds the error of its float solution a priori by
 * u (kappa + kappa^2 ||r|| / (||R|| ||p||)) with u = 2^-24, kappa <= ||R||_F ||R^{-1}||_F,
 * ||R|| kappa^2 <= ||R||_F ||R^{-1}||_F^2 and ||r|| from the bottom of Q^T b; blocks above the
 * selection threshold
 * (qrkit_set_refinement; 2e-6 by default) are refined by a second kernel with up to
 * `refine_steps` steps of Bjorck's iterative refinement of the augmented system
 * [I J_i; J_i^T 0] [r; p] = [b_i; 0] (not in the paper): from p_i and r = Q_i [0; c_i bottom],
 * each step takes f = b_i - r - J_i p_i and g = -J_i^T r in extended precision (compensated
 * float or double, qrkit_set_refinement), then h = R_i^{-T} g, [d1; d2] = Q_i^T f,
 * dp = R_i^{-1} (d1 - h), dr = Q_i [h; d2], p_i += dp, r += dr; a block stops once its
 * correction is below 1e-6 of its solution (max norms).  refine_steps is ignored for
 * QRKIT_FP32 and QRKIT_FP64.
 *   J    : packed values, block i column-major n_i x m_i, blocks in order (sum n_i m_i)
 *   b    : sum n_i values, block i's rows contiguous
 *   D    : with lambda > 0, sum m_i damping values or NULL for the column norms of J (zero ->
 *          1); ignored when lambda = 0
 *   lambda : >= 0.  lambda > 0 takes Moré's two factorizations (Sec. 5.2, Eq. LMTwoStep): the
 *          undamped QR above (refine_steps ignored, no refinement: float accuracy in the
 *          float modes), then qrkit_more_solve's second factorization per block; every block
 *          needs n_i >= m_i.  (The composed path, qrkit_factor with lambda > 0, refines.)
 *   p    : out, sum m_i values
 *   qtb  : out or NULL; sum n_i values: Q_i^T b_i per block
 * The factor (reflectors below the diagonal, R on and above it, tau) stays in the context.
 * One kernel launch (two in FP32 refined mode or with lambda > 0; banded plans: the banded
 * factor + solve and its refinement); asynchronous on the context's stream. */
qrkit_status qrkit_factor_solve(qrkit_ctx* ctx, const void* J, const void* b, const void* D,
                                double lambda, void* p, void* qtb, int refine_steps);

/* Poll limit of the bounded device waits (no paper counterpart): the tile mapping of the block
 * solve waits for its bulk copies on an mbarrier at most this many polls (default 2^26).  A
 * wait that runs out records QRKIT_ETIMEOUT in the device status word (qrkit_sync_status);
 * the kernel then waits for its own copies in flight with a limit of its own (2^26 polls)
 * before it returns, so no kernel traps or hangs and the context stays usable.  A small limit
 * (down to 0) makes the waits run out on purpose, which tests that failure path without a
 * GPU fault.  QRKIT_EINVAL for polls < 0. */
qrkit_status qrkit_set_wait_limit(qrkit_ctx* ctx, int64_t polls);

/* Moré's second factorization (Sec. 5.2, Eq. LMTwoStep) for the block-diagonal factor of the
 * last qrkit_factor_solve: with J_i = Q_i R_i kept, each damping value needs only, per block,
 * the QR of [R_i; lambda^(1/2) D_i] with the damping row of column k placed after row k of
 * R_i (the interleave of Sec. 4.5) and R'_i p_i = top of Q'_i^T [c_i; 0], c_i = the top m_i
 * entries of Q_i^T b_i.  Since ||J_i p - b_i||^2 = ||R_i p - c_i||^2 + const, p_i minimises
 * ||J_i p - b_i||^2 + lambda ||D_i p||^2 (Eq. 2).  Call it once per damping value of an LM
 * iteration (rejected steps cost only this).
 *   qtb    : DEVICE, sum n_i values: the Q^T b that qrkit_factor_solve wrote (lambda = 0)
 *   D      : DEVICE, sum m_i values, or NULL for the column norms of J (computed as those of
 *            R_i, equal since Q_i is orthogonal; zero -> 1)
 *   lambda : >= 0 (0 gives the undamped solution again)
 *   p      : DEVICE out, sum m_i values
 * One thread per block, the stack reduced by 2 x 2 reflections of the damping row against the
 * rows of R_i; no refinement.  A zero pivot is reported as QRKIT_ESINGULAR in the device status
 * word.  Asynchronous. */
qrkit_status qrkit_more_solve(qrkit_ctx* ctx, const void* qtb, const void* D, double lambda, void* p);

/* Moré's trust-region choice of the damping for the two-factorization step (Sec. 5.2, after
 * Moré 1977): the lambda >= 0 whose step p(lambda) (qrkit_more_solve's) has scaled length
 * ||D p|| within sigma delta of delta, or lambda = 0 when the undamped step is already that
 * short.  Each iteration is one stage 2 over all blocks that also sums ||D p||^2 and ||z||^2
 * (R'^T z = D^2 p, so d||D p||/dlambda = -||z||^2 / ||D p||); lambda moves by Newton's step on
 * 1/||D p|| - 1/delta inside a bracket that each iterate narrows (upper end
 * ||D^{-1} J^T b|| / delta).
 *   qtb, D, p     : as for qrkit_more_solve (D NULL: the column norms of J)
 *   delta         : > 0, the trust-region radius in the scaled norm
 *   sigma         : in (0, 1), the accepted relative deviation (0.1 is customary)
 *   max_iter      : >= 1
 *   lambda        : HOST out, the damping found
 *   iterations    : HOST out or NULL, stage-2 passes after the undamped one
 * p holds the step for the returned lambda.  QRKIT_ENOTCONV when max_iter passes do not
 * reach the tolerance (p and lambda then hold the last iterate); QRKIT_ESTATE without a
 * block-diagonal factor.  Synchronous (three sums are read back per iteration). */
qrkit_status qrkit_more_trust_region(qrkit_ctx* ctx, const void* qtb, const void* D, double delta, double sigma,
                                     int max_iter, double* lambda, void* p, int* iterations);

/* Result record of qrkit_get_info. */
typedef struct qrkit_info {
  int32_t refine_steps_max;   /* most refinement steps a block took in the last FP32-refined
                                 qrkit_factor_solve (warp-task mapping), else -1 */
  int64_t refined_blocks;     /* blocks its a-priori estimate selected, else -1 */
  double residual_norm;       /* ||b - J p||_2 */
  double optimality_norm;     /* ||J^T (b - J p) - lambda D^2 p||_2 */
  double optimality_scale;    /* ||J||_F (||J||_F ||p|| + ||b||): the size of J^T b and of
                                 J^T J p, against which optimality_norm is small */
} qrkit_info;

/* Diagnostics of a solution p of a block-diagonal plan (no paper counterpart; the quantities
 * are those of Eq. 1 and Eq. 2): the residual norm, the norm of the optimality residual
 * J^T (b - J p) - lambda D^2 p, which is zero at the exact minimiser of Eq. 2 ((J^T J +
 * lambda D^2) p = J^T b, Eq. 1), its scale, and the refinement's selection count and most steps
 * taken in the last qrkit_factor_solve.  J, b, p: DEVICE buffers as for qrkit_factor_solve; D:
 * DEVICE (sum m_i) or NULL for the column norms of J (zero -> 1); lambda >= 0.  Everything in
 * double, added in a fixed order.  Synchronous. */
qrkit_status qrkit_get_info(qrkit_ctx* ctx, const void* J, const void* b, const void* p, const void* D,
                            double lambda, qrkit_info* out);

/* Residual precision of the block refinement (qrkit_set_refinement). */
enum { QRKIT_RESIDUAL_DOT2 = 0, QRKIT_RESIDUAL_FP64 = 1 };

/* Settings of the FP32-refined block solve of qrkit_factor_solve (refinement is not in the
 * paper; its goal, single precision without the accuracy loss, is that of Sec. 1 and 7):
 *   select   : a block is refined when its a-priori error estimate exceeds this (in [0, 1];
 *              0 refines every block; default 2e-6)
 *   residual : QRKIT_RESIDUAL_DOT2 (default) computes the refinement's residuals as
 *              unevaluated float pairs by error-free transformations (Dot2), about as accurate
 *              as twice the float precision; QRKIT_RESIDUAL_FP64 computes them in double
 * Takes effect at the next qrkit_factor_solve; QRKIT_EINVAL for values outside these. */
qrkit_status qrkit_set_refinement(qrkit_ctx* ctx, double select, int residual);

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
 * refine_steps > 0: keep them alive and unchanged until then.  Dense S: s <= 64, or in the
 * float modes any multiple of 32 up to 512 (the reduced block is then blocked by column panels
 * of 32, Sec. 2: each panel a TSQR of its own, its Q^T applied to the later columns on the
 * tensor cores, 3xTF32 with float accumulation).  QRKIT_EUNSUPPORTED otherwise. */
qrkit_status qrkit_factor(qrkit_ctx* ctx, const void* J, const void* S, const void* D, double lambda);

/* qtb = Q^T [b; 0] restricted to its top N entries (Sec. 5.1, matrixQ().transpose() * b),
 * laid out as [c_blocks (sum m_i, column order) ; c_S (s)].  b: sum n_i values. */
qrkit_status qrkit_apply_qt(qrkit_ctx* ctx, const void* b, void* qtb);

/* p = R^{-1} qtb (Sec. 5.1, matrixR().solve): qtb as produced by qrkit_apply_qt; p: N values
 * (block columns then shared columns). */
qrkit_status qrkit_solve_r(qrkit_ctx* ctx, const void* qtb, void* p);

/* Sec. 5.1 (Q^T b, then the R solve) with refinement (not in the paper):
 * p = argmin ||P_r [J; lambda^(1/2) D] p - P_r [b; 0]|| with the stored factor: Q^T b,
 * back-substitution, then `refine_steps` refinement steps (QRKIT_FP32_REFINED: residual
 * g = J^T (b - J p) - lambda D^2 p in double, correction R^{-1} R^{-T} g; ignored for
 * QRKIT_FP32, allowed but not useful for QRKIT_FP64). */
qrkit_status qrkit_solve(qrkit_ctx* ctx, const void* b, void* p, int refine_steps);

/* ---- A dense S split by rows over several contexts (one per GPU): the horizontal
 * concatenation of Sec. 4.2 with the reduced shared block factored by TSQR across GPUs.  Each
 * context plans its own blocks and their rows of S, factors them with the global D (the shared
 * columns' damping entries set to zero, so that those rows enter once, at the merge), and
 * reports its s x s triangle R_g and c_g (the last s entries of qrkit_apply_qt); the stacked
 * [R_1; c_1 .. R_G; c_G; lambda^(1/2) D_S; 0] is solved once by qrkit_dense_lstsq, and each
 * context finishes its block unknowns with qrkit_solve_blocks. ---- */

/* Squared column sums of J = [blkdiag(J_i) | S] (DEVICE out, N doubles), added in a fixed
 * order: summed over contexts they give the global column norms (Sec. 5.2 D = diag(J^T J)^(1/2)).
 * Asynchronous. */
qrkit_status qrkit_column_sumsq(qrkit_ctx* ctx, const void* J, const void* S, double* sq);

/* D = sqrt(sq), zero -> 1 (Sec. 5.2, the MINPACK convention for a zero column), n values, D in
 * the context precision (DEVICE).  Asynchronous. */
qrkit_status qrkit_norms_from_sumsq(qrkit_ctx* ctx, const double* sq, int64_t n, void* D);

/* The s x s upper triangle R_S of the reduced shared block of the last qrkit_factor on a dense-S
 * plan (Sec. 4.2 Q_1-perp^T A_2 factored by TSQR), DEVICE out, column-major, zeros below the
 * diagonal.  Asynchronous. */
qrkit_status qrkit_get_reduced_r(qrkit_ctx* ctx, void* R);

/* The block unknowns for given shared unknowns (Sec. 5.1 back-substitution, the reduced solve
 * left out): qtb as from qrkit_apply_qt; p (DEVICE, N values) holds the shared unknowns in its
 * last s entries on entry and receives the block unknowns R_i^{-1} (c_i - R12_i p_S) in its first
 * sum m_i entries.  Asynchronous. */
qrkit_status qrkit_solve_blocks(qrkit_ctx* ctx, const void* qtb, void* p);

/* min ||A x - b|| for a dense A (DEVICE, M x N column-major, leading dimension lda, M >= N) by
 * Householder QR (Sec. 2) in one CTA, in the context precision; A and b are not changed.
 * res2 (HOST, may be NULL; the call then waits for the stream) receives ||b - A x||^2.  For the
 * merge of distributed triangles: N <= 1024 and M N <= 2^24 (QRKIT_EUNSUPPORTED beyond).
 * A zero pivot is reported as QRKIT_ESINGULAR in the device status word. */
qrkit_status qrkit_dense_lstsq(qrkit_ctx* ctx, int64_t M, int64_t N, const void* A, int64_t lda, const void* b,
                               void* x, double* res2);

/* Comparison path (Sec. 1, Sec. 6.1 "QRkit+Chol"): p from the normal equations Eq. (1),
 * (J^T J + lambda D^2) p = J^T b, by Cholesky in the context's precision (float for both float
 * modes; no refinement), for a QRKIT_STRUCT_BLOCKS plan of any coupling.  The block unknowns
 * are eliminated first (Schur complement onto the shared block, banded per segment for
 * windows, dense for a dense S with s <= 64).  Its error grows with cond(A)^2, the QR path's
 * with cond(A).  J, S, b, D, lambda, p as for qrkit_factor / qrkit_solve (D NULL: column
 * norms, zero -> 1).  A non-positive pivot is reported as QRKIT_ESINGULAR in the device
 * status word.  Asynchronous. */
qrkit_status qrkit_normal_solve(qrkit_ctx* ctx, const void* J, const void* S, const void* b, const void* D,
                                double lambda, void* p);

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
 * The work runs in the tile kernel (tiles of consecutive blocks, refinement inside the kernel),
 * not in the warp-task kernels the context path uses by default; the problem solved is the same.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current.  Every call is synchronous (it waits for its stream and copies the
 * status word back), so no call may be made while any stream is being captured.  The caller
 * thread's current device is the same after the call as before it.  `stream` must belong to
 * `device` (QRKIT_EINVAL otherwise).  Each call copies the shapes and schedule into the array,
 * clears its status word, launches one kernel on `stream`, then waits for the stream and reads
 * the status word back: every call, the first included, returns only after its work is done,
 * with the kernel's status (QRKIT_OK, QRKIT_ESINGULAR, ...).
 * Every call uses the same array and leaves its contents behind: calls whose work overlaps on
 * the GPU (other threads, other streams) race and must be serialized by the caller.  The
 * factor is not kept for later calls. */
qrkit_status qrkit_block_solve_noalloc(int device, void* stream, int precision,
                                       int64_t num_blocks, const uint8_t* block_rows,
                                       const uint8_t* block_cols, const void* J, const void* b,
                                       void* p, int refine_steps);

/* Banded factor (Sec. 4.4) of the last qrkit_factor_solve on a QRKIT_STRUCT_BANDED plan (device pointers,
 * any may be NULL): Rw[j * w + t] = R[j, j + t] per global column j, c = top of Q^T [b; 0] per
 * column; res2 (HOST, one double per instance) = squared residual norm.  Synchronous.
 * Rw and c exist only for the SWEEP algorithm (QRKIT_EUNSUPPORTED otherwise); res2 always. */
qrkit_status qrkit_get_band_factor(qrkit_ctx* ctx, void* Rw, void* c, double* res2);

/* Copy the stored factor of a block structure (Sec. 4.1; reflectors as in Sec. 2) to caller
 * buffers (device pointers, either may be NULL): factor values in J's packing (V strictly below
 * the diagonal, R on and above) and tau (sum m_i).  The warp-task solve keeps its factor in a
 * task-ordered layout of its own (whole 16-byte row quads, so that it is written in full
 * sectors); this call rearranges it with one kernel.  Asynchronous. */
qrkit_status qrkit_get_factor(qrkit_ctx* ctx, void* factor_out, void* tau_out);

/* Replace the window starts (Sec. 4.2 windows, re-sorted by the P_r of Sec. 4.3) of a
 * QRKIT_COUPLED_WINDOW plan from DEVICE memory (K int32, same
 * meaning as qrkit_structure.window_start), e.g. when an LM iteration moves the windows.
 * Copied asynchronously; a start outside its block's segment is clamped into it and
 * reported as QRKIT_EINVAL through the device status word.  Takes effect at the next
 * qrkit_factor. */
qrkit_status qrkit_set_window_start(qrkit_ctx* ctx, const int32_t* start);

/* Row permutation P_r of the reduced shared block of the last qrkit_factor on a windowed plan
 * (Sec. 4.3): order[k] = index of the reduced row at sorted position k (DEVICE, int64, one per
 * reduced row).  Reduced rows are numbered block by block, rows of a block in order (n_i rows
 * per block with damping, n_i - m_i without); the sort key is (segment, first S column,
 * reduced-row index).  Asynchronous. */
qrkit_status qrkit_get_row_order(qrkit_ctx* ctx, int64_t* order);

/* Autotuning (no paper counterpart): times candidate launch configurations for the current
 * plan on the given inputs (DEVICE buffers as for qrkit_factor_solve; p is overwritten) and
 * keeps the fastest.  Block plans without coupling: the block-to-warp mapping of the fused
 * solve, "tasks <supertile> <warps per CTA> [<key-major 0/1>]" (shape-uniform warp tasks, the
 * default; see qrkit_task_layout) or
 * "budget <blocks> <values> <rows> <cols> <padded>" (tiles of consecutive blocks); parallel
 * banded plans: the compression strategy "compress <thread rows 0/1> <splits>" (one thread per
 * column block, or warps with 1-8 splits).  cache_path (HOST string, may be NULL): a text file with one line per
 * structure key (GPU name, precision, shape signature) and its choice; a key found there is
 * applied without timing, a new choice is appended.  chosen (HOST, may be NULL): receives the
 * choice as text.  Synchronous. */
qrkit_status qrkit_autotune(qrkit_ctx* ctx, const void* J, const void* b, void* p, int refine_steps,
                            const char* cache_path, char* chosen, int64_t chosen_len);

/* Apply a configuration in the text form qrkit_autotune returns (HOST string; no paper
 * counterpart) to the current plan without timing, e.g. one chosen earlier on the same GPU.  QRKIT_EINVAL if the text does
 * not parse or does not fit the plan's kind; synchronous. */
qrkit_status qrkit_apply_tuning(qrkit_ctx* ctx, const char* choice);

/* The warp tasks a block plan (QRKIT_STRUCT_BLOCKS, QRKIT_COUPLED_NONE) hands to the fused
 * solve of Sec. 4.1, computed on the host with no CUDA call and no context, for inspection
 * and tests.  The blocks are taken in supertiles of `supertile` consecutive blocks (32..65536;
 * qrkit_plan uses 65536); inside a supertile they are sorted, stably, by shape key
 * 8 * ((n_i - 1) / 4) + (m_i - 1), and each key's run is cut into tasks of P blocks, where
 * P = 32 / G and G = (n_i - 1) / 4 + 1 lanes of a warp hold one block (P = 32, 16, 10, 8); only
 * the last task of a run has unused slots.  Tasks are in supertile order, keys ascending
 * inside a supertile; key_major != 0 reorders them stably by key.
 *   block_rows, block_cols : HOST, num_blocks shapes as in qrkit_structure (1..16, 1..8)
 *   num_tasks              : HOST out: the number of tasks
 *   task_key               : HOST out or NULL: the key of each task
 *   task_slots             : HOST out or NULL: int64[num_tasks][32][4]: per task and slot the
 *                            block index and its first value, row and column (offsets into
 *                            J's packing, b and p); -1 in all four for an unused slot
 *   capacity               : tasks the out arrays hold
 * With task_key and task_slots both NULL only num_tasks is set.  QRKIT_EINVAL for a bad
 * argument or a capacity below num_tasks (num_tasks is still set), QRKIT_EUNSUPPORTED for a
 * shape outside 16 x 8. */
qrkit_status qrkit_task_layout(int64_t num_blocks, const uint8_t* block_rows, const uint8_t* block_cols,
                               int64_t supertile, int key_major, int64_t* num_tasks, int32_t* task_key,
                               int64_t* task_slots, int64_t capacity);

/* In/out record of qrkit_structure_metadata. */
typedef struct qrkit_metadata {
  int32_t damped;       /* in */
  int64_t num_blocks;   /* out */
  int64_t rows;         /* out: J rows (sum n_i) */
  int64_t cols;         /* out: N = sum m_i + shared columns */
  int64_t values;       /* out: sum n_i m_i */
  int64_t aug_rows;     /* out: rows of [J; lambda^(1/2) D] (rows, plus cols when damped) */
  int64_t* val_off;     /* HOST out or NULL */
  int64_t* row_off;     /* HOST out or NULL */
  int64_t* col_off;     /* HOST out or NULL */
  int64_t* row_order;   /* HOST out or NULL */
  int64_t* r_row_ptr;   /* HOST out or NULL */
  int32_t* r_col_idx;   /* HOST out or NULL */
  int64_t r_capacity;   /* in: entries r_col_idx holds */
  int64_t r_nnz;        /* out: entries of the R pattern (-1 if not asked for) */
} qrkit_metadata;
/* Structure metadata of a QRKIT_STRUCT_BLOCKS descriptor (Sec. 3 composition, Sec. 4.5 / 5.2
 * row interleave), on the host with no CUDA call and no context.  in: damped (1: the damping
 * rows lambda^(1/2) D are present, i.e. lambda > 0).  out: the sizes; and, where the HOST
 * pointers are not NULL, the offsets of the packed values, rows and columns of each block
 * (num_blocks + 1 each), the row permutation P_r of [J; lambda^(1/2) D] (aug_rows entries: the
 * source row of each row, J rows 0 .. rows - 1, the damping row of column j = rows + j; sorted by
 * leading column, J rows before the damping row of that column, then by source index) and the
 * structural pattern of R in natural column order (block columns, then shared columns) as CSR:
 * r_row_ptr (cols + 1) and r_col_idx (r_nnz entries, columns ascending per row; r_capacity
 * entries available).  The pattern is that of the row-merge QR of the rows in P_r order (a row
 * whose leading column c already has an R row is merged with it, both taking the union of the
 * two patterns), which is the pattern of the unique R barring cancellation.  A window is cut at
 * the end of its block's segment.  QRKIT_EINVAL for a malformed descriptor or too small a
 * capacity (r_nnz is still set), QRKIT_EUNSUPPORTED for other structure kinds. */
qrkit_status qrkit_structure_metadata(const qrkit_structure* s, qrkit_metadata* md);

/* Row and column permutations that expose a banded structure (Sec. 4.3), on the host with no
 * CUDA call: P_c by reverse Cuthill-McKee on the column graph of A (columns adjacent when a row
 * holds both; each search starts at the unvisited column of least degree, lower index first;
 * neighbours are queued by (degree, index); the visit order is reversed), P_r by the rows'
 * (first, last) column under P_c, ties by row index, empty rows last.
 *   rows, cols        : shape of A (cols >= 1)
 *   row_ptr, col_idx  : HOST, the pattern in CSR form (rows + 1 offsets from 0; column indices
 *                       in [0, cols), any order, repeats allowed)
 *   col_perm          : HOST out, cols entries: original column at each new position
 *   row_perm          : HOST out, rows entries: original row at each new position
 *   row_start         : HOST out, rows entries: first new column of that row (cols if empty)
 *   width             : HOST out: band width w; row k of P_r A P_c lies in columns
 *                       row_start[k] .. row_start[k] + w - 1
 * QRKIT_EINVAL for a malformed pattern.  Synchronous; O(sum over rows of nnz(row)^2) time. */
qrkit_status qrkit_band_order(int64_t rows, int64_t cols, const int64_t* row_ptr, const int32_t* col_idx,
                              int32_t* col_perm, int64_t* row_perm, int32_t* row_start, int32_t* width);

/* ---- Levenberg-Marquardt on the device (Sec. 2; Backtrack LM of Sec. 5.2) ----
 * Model QRKIT_MODEL_CURVEFIT: 2-D points fitted by an open uniform cubic B-spline; each
 * point has one latent curve parameter t_i and the control points are shared, so J is
 * block-angular with 2x1 blocks and, per point, a window of 8 shared columns (Sec. 4.2 with
 * the banded reduced block of Sec. 4.4; the shape of the paper's surface fits, Sec. 6.2).
 *   seg = clamp(floor(t), 0, Kc - 4), u = t - seg,
 *   curve(t) = sum_{q=0..3} B_q(u) P_{seg+q} with the uniform cubic B-spline basis
 *   B_0 = (1-u)^3/6, B_1 = (3u^3 - 6u^2 + 4)/6, B_2 = (-3u^3 + 3u^2 + 3u + 1)/6, B_3 = u^3/6,
 *   f_i = curve(t_i) - data_i (two rows per point), cost = 1/2 ||f||^2.
 * Several independent problems are solved together (one segment of S each). */
typedef enum { QRKIT_MODEL_CURVEFIT = 0 } qrkit_model;

typedef struct qrkit_lm_problem {
  int32_t model;                 /* QRKIT_MODEL_CURVEFIT */
  int64_t num_problems;          /* B >= 1 */
  const int64_t* num_points;     /* host, B entries >= 1: P_k */
  const int32_t* control_points; /* host, B entries >= 4: Kc_k */
  const double* data;            /* DEVICE, (sum P_k) x 2 doubles (x, y), problems in order;
                                    read by every step: keep it alive and unchanged */
} qrkit_lm_problem;

/* Per-problem LM state (host structs; copied to the device and back by each call). */
typedef struct qrkit_lm_state {
  double lambda;     /* in/out: damping, > 0 */
  double nu;         /* in/out: Nielsen's growth factor after a rejection (start with 2) */
  double cost;       /* out: 1/2 ||f(x)||^2 at the start of the last step */
  double cost_new;   /* out: 1/2 ||f(x + p)||^2 of the last trial */
  double pred;       /* out: predicted decrease 1/2 p^T (lambda D^2 p + J^T b), b = -f */
  double rho;        /* out: gain ratio (cost - cost_new) / pred; -1 when pred <= 0 */
  int32_t accepted;  /* out: the last trial was taken (rho > 0) */
  int32_t done;      /* in/out: 1 = stopped; a stopped problem no longer changes */
  int64_t iteration; /* in/out: steps tried */
} qrkit_lm_state;

/* Plan the LM model (Sec. 2, Sec. 5.2; the curve-fit model is ours): builds the block-angular structure (2x1 blocks, windows of 8, one
 * segment per problem, replacing the context's plan) and the device buffers.  x, passed to
 * the calls below, is a DEVICE array of N = sum P_k + sum 2 Kc_k doubles:
 * [t of all points, problems in order | control points of problem 0 (x0, y0, x1, y1, ...),
 * problem 1, ...].  Synchronous. */
qrkit_status qrkit_lm_plan(qrkit_ctx* ctx, const qrkit_lm_problem* problem);

/* One LM iteration (Sec. 2; Backtrack LM of Sec. 5.2) for every problem not marked done: f, J and the window starts at x;
 * D = column norms of J (zero -> 1); QR of P_r [J; lambda^(1/2) D] by the composed path with
 * the rows of J, S and b rounded to the context precision; p from qrkit_solve with
 * `refine_steps`; cost at x + p; gain ratio; Nielsen update (rho > 0: accept,
 * lambda *= max(1/3, 1 - (2 rho - 1)^3), nu = 2; else lambda *= nu, nu *= 2); x += p where
 * accepted.  A problem whose lambda exceeds 1e16 is marked done.  states: host, B entries,
 * read and written.  Synchronous (returns after the state is copied back). */
qrkit_status qrkit_lm_step(qrkit_ctx* ctx, double* x, qrkit_lm_state* states, int refine_steps);

/* One LM trial step for a model of the caller's own (Sec. 2; Backtrack LM of Sec. 5.2): the
 * caller evaluates its residual f and Jacobian at x and passes J, S (the layout of
 * qrkit_factor for the current QRKIT_STRUCT_BLOCKS plan) and b = -f; the library factors
 * P_r [J; lambda^(1/2) D] (D NULL: column norms of J, zero -> 1), solves with `refine_steps`
 * refinement steps into p (DEVICE, N values) and returns in *pred (HOST) the predicted decrease
 * 1/2 p^T (lambda D^2 p + J^T b) of the linear model, computed in double.  The caller then
 * evaluates cost_new = 1/2 ||f(x + p)||^2 and forms the gain ratio rho = (cost - cost_new) /
 * pred for qrkit_nielsen_update.  J and S stay in use until the call returns.  Synchronous. */
qrkit_status qrkit_lm_trial(qrkit_ctx* ctx, const void* J, const void* S, const void* b, const void* D,
                            double lambda, int refine_steps, void* p, double* pred);

/* Nielsen's damping rule (the reading of the paper's "adapting Lourakis", Sec. 2 / Sec. 5.2):
 * rho > 0: the step is accepted, lambda *= max(1/3, 1 - (2 rho - 1)^3), nu = 2; otherwise
 * rejected, lambda *= nu, nu *= 2.  HOST values, read and written; accepted (may be NULL)
 * receives 1 or 0.  QRKIT_EINVAL unless lambda > 0 and nu > 0.  No CUDA call. */
qrkit_status qrkit_nielsen_update(double rho, double* lambda, double* nu, int32_t* accepted);

/* Up to max_iter iterations as in qrkit_lm_step (Sec. 2, Sec. 5.2) with the state kept on the device; a problem
 * is marked done after an accepted step with cost - cost_new <= ftol * cost (or lambda > 1e16),
 * and the loop ends early once every problem is done (checked every 8 iterations).  With
 * use_graph != 0 one iteration is captured into a CUDA graph (on the first call, or when x,
 * ftol or refine_steps change) and replayed; capture needs the context's stream to be a
 * stream other than the legacy default stream.  Synchronous. */
qrkit_status qrkit_lm_run(qrkit_ctx* ctx, double* x, qrkit_lm_state* states, int max_iter, double ftol,
                          int refine_steps, int use_graph);

/* The linearised system (Sec. 2; block-angular as in Sec. 4.2) of the planned LM model at x
 * (DEVICE buffers, any may be NULL), in the
 * layout of a QRKIT_COUPLED_WINDOW block structure with window 8: J (2 x 1 block per point,
 * 2 sum P_k values), S (per point 2 x 8 column-major, 16 sum P_k values), b = -f (2 sum P_k),
 * all in the context precision, and the window starts (int32, sum P_k; global shared column).
 * Asynchronous. */
qrkit_status qrkit_lm_linearize(qrkit_ctx* ctx, const double* x, void* J, void* S, void* b, int32_t* start);

/* Residual (Sec. 2) of the planned LM model at x: f (DEVICE, 2 sum P_k doubles) = curve(t_i) - data_i
 * per point, (x, y) pairs.  Asynchronous. */
qrkit_status qrkit_lm_residual(qrkit_ctx* ctx, const double* x, double* f);

/* ---- Learned damping (not in the paper; Nielsen's rule stays the fallback) ----
 * A 3-layer MLP, QRKIT_MLP_FEATURES -> 64 -> 64 -> QRKIT_MLP_CLASSES (ReLU), whose classes are
 * lambda multipliers {1e-2, 1e-1, 1/3, 1/2, 1, 2, 4, 10}.  With the policy on, an LM step that
 * is accepted sets lambda_next = lambda * multiplier[argmax]; a rejected step uses Nielsen's
 * rule (lambda *= nu, nu *= 2).  Features of problem k after each step (float32, in order):
 * log10(lambda) / 4, log10(iteration + 1) / 2, gain ratios of the last 4 steps (clamped to
 * [-1, 2], newest first), their acceptance flags (0/1), log10(cost_new / cost) of the last 4
 * steps clamped to [-8, 1] / 8, log10(pred / cost) clamped to [-16, 0] / 16, and 1.
 * Parameters: QRKIT_MLP_PARAMS float32 values [W1 (64 x 16) | b1 | W2 (64 x 64) | b2 |
 * W3 (8 x 64) | b3], row-major; the forward and backward passes use the weight matrices
 * rounded to bfloat16 (round to nearest even) with float32 accumulation; Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8) updates the float32 copy.  The MLP belongs to the context. */
#define QRKIT_MLP_FEATURES 16
#define QRKIT_MLP_CLASSES 8
#define QRKIT_MLP_PARAMS 5768

/* Set the MLP parameters (HOST, QRKIT_MLP_PARAMS floats) and reset Adam.  Synchronous.  (Not
 * in the paper.) */
qrkit_status qrkit_mlp_init(qrkit_ctx* ctx, const float* params);

/* Copy the current float32 parameters to HOST memory.  Synchronous.  (Not in the paper.) */
qrkit_status qrkit_mlp_params(qrkit_ctx* ctx, float* params);

/* logits (DEVICE, n x QRKIT_MLP_CLASSES) of the samples X (DEVICE, n x QRKIT_MLP_FEATURES).
 * (Not in the paper.) */
qrkit_status qrkit_mlp_forward(qrkit_ctx* ctx, const float* X, int64_t n, float* logits);

/* One training step on a batch (not in the paper): mean softmax cross-entropy of X (DEVICE, n x FEATURES) against
 * labels (DEVICE int32, n, in [0, CLASSES)), its gradient, and (lr > 0) an Adam update.
 * loss (HOST, may be NULL; synchronous when given), grad (DEVICE, QRKIT_MLP_PARAMS, may be
 * NULL): the loss and gradient at the parameters before the update. */
qrkit_status qrkit_mlp_train_step(qrkit_ctx* ctx, const float* X, const int32_t* labels, int64_t n, float lr,
                                  float* loss, float* grad);

/* Damping of the planned LM model: 0 = Nielsen's rule (Sec. 2 adapting Lourakis, Sec. 5.2),
 * 1 = the context's MLP after accepted steps (not in the paper; Nielsen after rejected ones). */
qrkit_status qrkit_lm_set_policy(qrkit_ctx* ctx, int use_mlp);

/* Features of every problem after the last LM step (DEVICE, B x QRKIT_MLP_FEATURES floats).
 * (Not in the paper.) */
qrkit_status qrkit_lm_features(qrkit_ctx* ctx, float* features);

/* Peak-rate probe of a device (no paper counterpart; the roofline denominators no library
 * measures): kind 0 = FP32 fused multiply-add throughput of the CUDA cores, 1 = FP64 FMA,
 * 2 = dense TF32 rate of the tensor cores (tcgen05.mma kind::tf32, M = 128, N = 256, FP32
 * accumulation).  *tflops (HOST) receives the rate in TFLOP/s (2 flops per multiply-add) of
 * the second of two timed launches over every SM.  Allocates 64 bytes and a stream of its own;
 * the caller thread's current device is restored.  Synchronous. */
qrkit_status qrkit_peak_probe(int device, int kind, double* tflops);

/* Host-link probe of a device (no paper counterpart; it explains the end-to-end rate of a solve
 * whose inputs start in host memory): `bytes` (>= 1 MiB, a multiple of 16) of pinned host memory
 * moved to device memory by cudaMemcpyAsync (*copy_gbs) and by a kernel that reads the pinned
 * memory directly (*kernel_gbs), in GB/s, each the second of two timed runs.  Allocates its own
 * host and device buffers and a stream; the caller thread's current device is restored.
 * Synchronous. */
qrkit_status qrkit_host_link_probe(int device, int64_t bytes, double* copy_gbs, double* kernel_gbs);

/* Block until the stream is idle and return the device status word (QRKIT_OK if no kernel
 * reported a failure), then clear it.  (No paper counterpart.) */
qrkit_status qrkit_sync_status(qrkit_ctx* ctx);

/* Number of this library's kernels launched on ctx since creation (for launch accounting; no
 * paper counterpart). */
int64_t qrkit_launch_count(const qrkit_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* QRKIT_H */
