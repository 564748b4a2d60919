// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qrkit.h"

namespace qrkit {

// Device status word values mirror qrkit_status.  Kernels record the first failure with
// atomicCAS and never trap.
constexpr int kDevOk = QRKIT_OK;

// Tile budgets of the persistent block kernels (one tile = consecutive blocks staged in
// shared memory; the plan cuts tiles greedily so no budget is exceeded).
struct TileBudget {
  int blocks;   // blocks per tile
  int values;   // J values per tile
  int rows;     // J rows per tile
  int cols;     // columns per tile
  int padded;   // padded working-area values per tile (rows rounded up to 4, 8 or 16)
};

// Warp tasks of the batched block solve (block_tasks.cu).  A task is P = floor(32 / G)
// blocks of one shape key (row class c = (n - 1) / 4, column count m; key = 8 c + m - 1),
// G = c + 1 lanes per block; entries are relative to the task's supertile bases.
constexpr int kTaskKeys = 32;
struct TaskHdr {
  int64_t v0, r0, c0, b0;   // value, row, column and block offsets of the supertile
  int64_t first;            // first of the task's P entries
  int32_t key;
  int32_t plane;            // first of the task's M planes of the stored factor (see below)
};
// The factor the warp-task kernels keep: per task M planes of kPlaneValues values, plane j =
// column j of the task's blocks, block slot s at s * 4G, rows 4q .. 4q + 3 of lane q of its
// group at 4q (rows past n are zero); tau in planes of kTauPlane values, tau_k of slot s at
// plane k, entry s.  Lanes store whole 16-byte row quads, so every plane is written in full.
constexpr int kPlaneValues = 128;
constexpr int kTauPlane = 32;
struct TaskEntry {
  uint32_t v, r, c;         // offsets relative to the supertile bases
  uint16_t blk;             // block index relative to the supertile
  uint8_t n, m;             // shape; n = 0 marks an unused entry
};
static_assert(sizeof(TaskHdr) == 48 && sizeof(TaskEntry) == 16, "task layout");

// A device buffer owned by the context.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Plan {
  bool valid = false;
  bool composed = false;  // coupled part present (or damping on a block structure)
  qrkit_structure s{};
  int64_t K = 0;          // blocks
  int64_t rows = 0;       // sum n_i (J rows)
  int64_t cols = 0;       // sum m_i (block columns)
  int64_t values = 0;     // sum n_i m_i
  int max_n = 0, max_m = 0;
  int64_t first_wide = -1;      // first block with n_i < m_i (needs damping rows), or -1
  int64_t first_tall_aug = -1;  // first block with n_i + m_i > 16 (no room for damping rows)
  // host copies
  std::vector<uint8_t> n, m;
  std::vector<int64_t> tile_block, tile_val, tile_row, tile_col;
  int64_t num_tiles = 0;
  TileBudget budget{};
  std::vector<int64_t> val_off, row_off, col_off;   // K + 1 each
  std::vector<int32_t> start;                      // window starts (QRKIT_COUPLED_WINDOW)
  // independent segments of the windowed S (one segment = all shared columns by default)
  std::vector<int64_t> seg_cols, seg_col0, seg_blocks, seg_blk0;   // seg_col0 / seg_blk0: nseg + 1
  // device copies
  DevBuf d_n, d_m, d_tile_block, d_tile_val, d_tile_row, d_tile_col;
  DevBuf d_val_off, d_row_off, d_col_off, d_start;
  DevBuf d_seg;   // 2 x (nseg + 1): seg_blk0 then seg_col0
  // warp tasks (uncoupled block plans): mapping 0 = warp tasks, 1 = tiles (block_solve.cu)
  int mapping = 0;
  int64_t supertile = 0;
  int task_warps = 8;                 // warps per CTA
  bool key_major = false;             // tasks ordered by shape key first
  int64_t num_tasks = 0;
  int64_t max_refine_tasks = 0;       // refinement tasks if every block were selected
  int64_t narrow_tasks = 0;           // float plans: tasks [0, narrow_tasks) hold blocks of <= 4 columns
  std::vector<int64_t> key_off;       // kTaskKeys + 1: blocks per key, prefix sums
  int64_t factor_planes = 0;          // planes of the stored factor (all tasks)
  std::vector<int64_t> rec_off;       // kTaskKeys + 1: offsets of the keys' refinement records
  DevBuf d_task_hdr, d_task_ent, d_key_off, d_rec_off;
};

// Read-only view of a block-angular structure and its values (device pointers).
template <typename T>
struct ComposedView {
  int64_t K;
  const uint8_t* n;
  const uint8_t* m;
  const int64_t* val_off;
  const int64_t* row_off;
  const int64_t* col_off;
  const int32_t* start;
  int coupled;
  int s;          // shared columns
  int w;          // coupled columns per block (s for dense S)
  int64_t rows;   // J rows (sum n_i), leading dimension of a dense S
  int64_t nb;     // block columns (sum m_i)
  const T* J;
  const T* S;
};

// Where the composed factor lives.
template <typename T>
struct FactorOut {
  bool damp;
  double lam_half;
  const double* D;
  T* Fa;
  T* tau;
  T* R12;
  T* ctop;
  const int64_t* aug_off;
  const int64_t* red_off;
  T* X0;
  int64_t ld0;
  T* Xw;            // windowed reduced rows (rows x w, row-major)
  int64_t* Xstart;  // their first column
  int* status;
};

struct CRPlan;   // parallel banded QR (cr.cu)
void release_cr(CRPlan*& p);

// Chunk tables of the device row sort of the windowed reduced block (Sec. 4.3 P_r).
struct RowSortTables {
  int64_t num_chunks;
  const int64_t* chunk_row0;   // first reduced row of the chunk
  const int64_t* chunk_rows;
  const int64_t* chunk_hoff;   // offset of the chunk's histogram (its segment's column count)
  const int64_t* chunk_col0;   // first shared column of the chunk's segment
  const int64_t* chunk_cols;   // shared columns of that segment
  const int64_t* chunk_out0;   // first sorted position of that segment
  const int64_t* seg_chunk0;   // nseg + 1: first chunk of each segment
};

// Device state of a batch of banded instances (Sec. 4.4).
struct Band {
  int64_t num_inst = 0, total_cols = 0, total_rows = 0;
  int rows_per_col = 1, w = 1;
  bool parallel = false;          // QRKIT_BAND_PARALLEL in effect
  bool explicit_starts = false;   // rows carry explicit starts (band_row_start)
  CRPlan* cr = nullptr;
  DevBuf d_cols, d_col0, d_row0, Rw, c, D, res2, g, h, r;
  DevBuf d_inst, d_rows, d_start;   // explicit starts: 4 x num_inst table, rows, global starts
};

struct TsqrLevel {
  int64_t M = 0;      // rows of the level matrix
  int64_t ld = 0;     // its leading dimension: M rounded up to a multiple of 4 (16-byte columns)
  int64_t tiles = 0;
  int64_t down0 = 0;  // column panels: first row of this level's retired rows in the next panel
  DevBuf X, tau, rhs;
  DevBuf T;           // column panels: the tiles' compact-WY T factors (32 x 32 per 32 columns)
};

// One column panel of a dense reduced block wider than one tile: columns [c0, c0 + pw) are
// factored by TSQR over the rows the earlier panels left, and the panel's Q^T is applied to
// the w - pw columns after it.
struct TsqrPanel {
  int c0 = 0, pw = 0, w = 0;
  std::vector<TsqrLevel> levels;
};

// Device state of the composed factorization.
struct Composed {
  bool damp = false;
  double lam = 0.0, lam_half = 0.0;
  int tile_rows = 256;
  int64_t red_rows = 0;            // stacked block bottoms
  int64_t aug_values_d = 0, aug_values_u = 0;
  int64_t red_rows_d = 0, red_rows_u = 0;
  DevBuf D, sq, Fa, tau, R12, ctop, g, h;
  DevBuf Xw, Xstart, rhs_red, RwS, cS, res2, meta;   // windowed reduced block
  // device row sort of the windowed reduced block, per damping state (-1: not built)
  int sort_damp = -1;
  int64_t sort_hist_entries = 0;
  RowSortTables sort{};
  DevBuf sort_tab, hist, spos, order, Xw_s, Xstart_s, rhs_s;
  DevBuf seg_inst;                 // 4 x nseg: cols, col0, row0, rows of the segments' banded solves
  CRPlan* cr = nullptr;            // parallel banded QR of the segments (window <= 8)
  // normal-equations (Cholesky) comparison path
  DevBuf nrm_D, nrm_L, nrm_W, nrm_y, nrm_As, nrm_rs, nrm_seg;
  DevBuf d_aug_off_d, d_aug_off_u, d_red_off_d, d_red_off_u;
  std::vector<TsqrLevel> levels;   // TSQR levels of the first (or only) column panel
  std::vector<TsqrPanel> panels;   // s > 128: the column panels after the first
  int panel0_w = 0;                // columns of the first panel's factor (s, or 128 with panels)
  DevBuf Rs, cs;                   // with panels: R_S (s x s, column-major) and its rhs
  DevBuf dense_ws;                 // qrkit_dense_lstsq: the copied matrix and rhs
  const void* J = nullptr;         // caller's values recorded at factor time
  const void* S = nullptr;
};

// Instance tables (host) -> level work lists and work space of the parallel banded QR.
qrkit_status cr_build(qrkit_ctx* ctx, CRPlan*& out, const std::vector<int64_t>& cols,
                      const std::vector<int64_t>& col0, const std::vector<int64_t>& row0,
                      const std::vector<int64_t>& rows);
// QR + solve of every instance: rows with explicit sorted starts (global columns) or
// implicit starts floor(i / rpc); damping rows lambda^(1/2) D_j; x and D by global column.
qrkit_status cr_solve(qrkit_ctx* ctx, CRPlan& C, const int64_t* starts, int rpc, int w, const void* J,
                      const void* b, const double* D, double lambda, void* x, double* res2);
// Compression strategy of the parallel banded QR: one thread per column block, or warps
// with `splits` splits per block (autotuning).
qrkit_status cr_set_strategy(qrkit_ctx* ctx, CRPlan& C, bool thread_rows, int splits);
// dx = R^{-1} R^{-T} g with the factor of the last cr_solve (g double, dx by global column).
qrkit_status cr_normal_solve(qrkit_ctx* ctx, CRPlan& C, const double* g, void* dx);

// Damping-policy MLP parameters and training state (mlp.cu)
struct Mlp {
  DevBuf theta, wbf, m, v, grad, partial, loss_part, loss;
  int64_t step = 0;
};
void release_mlp(Mlp*& m);

struct LM;   // Levenberg-Marquardt state of a planned model (lm.cu)
void release_lm(LM*& lm);

struct Workspace {
  DevBuf factor;   // factor values (J packing)
  DevBuf tau;      // sum m_i
  DevBuf rlist, rcount;   // blocks selected for refinement (4 row-class lists) and their counts
  DevBuf tlist, tcount;   // the same for the warp-task kernels (one list per shape key)
  DevBuf tfactor, ttau;   // factor and tau of the warp-task kernels in task planes
  DevBuf rrec;            // refinement records (J and b of the selected blocks)
  DevBuf qtb;             // Q^T b of a damped fused solve (Moré's stage 1)
};

}  // namespace qrkit

struct qrkit_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = QRKIT_FP32_REFINED;
  int num_sms = 0;
  size_t max_smem_optin = 0;
  std::string last_error;
  qrkit::Plan plan;
  qrkit::Workspace ws;
  qrkit::Composed comp;
  qrkit::Band band;
  qrkit::LM* lm = nullptr;    // LM model plan and buffers (qrkit_lm_plan)
  qrkit::Mlp* mlp = nullptr;  // damping-policy MLP (qrkit_mlp_init)
  int* d_status = nullptr;   // device status word
  int64_t launches = 0;
  size_t smem_attr[16] = {};   // dynamic smem opted in, per kernel variant (slot per kernel)
  int occ_threads[16] = {};    // threads and resident CTAs per SM at that size (warp-task kernels)
  int occ_per_sm[16] = {};
  long long wait_limit = 1LL << 26;  // polls of a bounded device wait before it gives up
  bool refine_stats = false;    // ws.tcount holds the last fused solve's selection counts and steps
  qrkit::DevBuf more_sums;      // trust-region lambda: the three block sums of an iteration
  float refine_select = 2e-6f;  // block refinement: a-priori error estimate that selects a block
  int refine_residual = 0;      // its residual precision: 0 compensated float, 1 double
  bool factored = false;       // fused block path
  bool factor_in_planes = false;  // the fused factor is in task planes (warp-task kernels)
  bool comp_factored = false;  // composed path
  bool band_factored = false;  // banded path
};

namespace qrkit {

qrkit_status fail(qrkit_ctx* ctx, qrkit_status st, const std::string& msg);
qrkit_status cuda_fail(qrkit_ctx* ctx, cudaError_t e, const char* what);
qrkit_status ensure(qrkit_ctx* ctx, DevBuf& buf, size_t bytes, const char* what);
void release(DevBuf& buf);
inline size_t elem_size(const qrkit_ctx* ctx) {
  return ctx->precision == QRKIT_FP64 ? sizeof(double) : sizeof(float);
}

// Tile schedule of the persistent block kernels (fills P.tile_* and P.num_tiles).
void cut_tiles_for(Plan& P);
TileBudget block_solve_budget(size_t elem);

// Launchers implemented in the kernel translation units.
qrkit_status composed_layout(qrkit_ctx* ctx, size_t elem);
qrkit_status widen_to_double(qrkit_ctx* ctx, const float* in, double* out, int64_t n);
qrkit_status composed_factor(qrkit_ctx* ctx, const void* J, const void* S, const void* D, double lambda);
// Composed factor with the damping diagonal given directly as E = lambda^(1/2) D (double,
// N entries) and lambda = 1: per-column damping, e.g. one lambda per independent problem.
qrkit_status composed_factor_scaled(qrkit_ctx* ctx, const void* J, const void* S, const double* E);
// D = column norms of the block structure's J (zero -> 1), N doubles.
qrkit_status composed_column_norms(qrkit_ctx* ctx, const void* J, const void* S, double* D);
template <typename T> ComposedView<T> composed_view(qrkit_ctx* ctx, const void* J, const void* S);
qrkit_status composed_solve(qrkit_ctx* ctx, const void* J, const void* S, const void* b, void* p,
                            int refine_steps);
qrkit_status composed_apply_qt(qrkit_ctx* ctx, const void* b, void* qtb);
qrkit_status composed_solve_r(qrkit_ctx* ctx, const void* qtb, void* p);
// Pieces of the dense-S solve split over several contexts (distributed TSQR).
qrkit_status composed_column_sumsq(qrkit_ctx* ctx, const void* J, const void* S, double* out);
qrkit_status composed_norms_from_sumsq(qrkit_ctx* ctx, const double* sq, int64_t n, void* D);
qrkit_status composed_reduced_r(qrkit_ctx* ctx, void* R);
qrkit_status composed_solve_blocks(qrkit_ctx* ctx, const void* qtb, void* p);
void release_composed(Composed& C);
qrkit_status banded_plan(qrkit_ctx* ctx, const qrkit_structure* s);
qrkit_status banded_factor_solve(qrkit_ctx* ctx, const void* J, const void* b, const void* D,
                                 double lambda, void* p, int refine_steps);
qrkit_status banded_get_factor(qrkit_ctx* ctx, void* Rw_out, void* c_out, double* res2_out);
// Banded factor + solve of num_inst instances whose rows have explicit starts (grouped per
// instance, non-decreasing within one); inst: 4 x num_inst device int64 (cols, col0, row0, rows).
qrkit_status banded_explicit_solve(qrkit_ctx* ctx, int64_t num_inst, const int64_t* inst,
                                   const void* rows, const int64_t* starts, const void* rhs, int w,
                                   const double* D, double lambda, void* Rw, void* c, void* x,
                                   double* res2);
qrkit_status banded_tri_solve(qrkit_ctx* ctx, int64_t num_inst, const int64_t* inst, const void* Rw,
                              int w, void* v, bool transpose);
qrkit_status reduced_row_sort(qrkit_ctx* ctx, const RowSortTables& t, int64_t nseg, int64_t hist_entries,
                              const int64_t* Xstart, const void* Xw, int w, int* hist, int64_t* spos,
                              int64_t* order, int64_t* Xstart_s, void* Xw_s);
qrkit_status window_start_copy(qrkit_ctx* ctx, const int32_t* in);
// One TSQR level of a 32-column panel (float, 256-row tiles, columns in registers): reflectors
// and R in place, tau per column, each tile's 32 x 32 T (Tout, optional), the R rows to Xn.
qrkit_status tsqr_panel_tile(qrkit_ctx* ctx, float* X, int64_t ld, int64_t M, float* taus, float* Xn, int64_t ldn,
                             int64_t tiles, float* Tout);
// Column-panel TSQR (float): the Q^T of every 256-row tile of a factored panel
// (reflectors in X's first pw columns, T factors from tsqr_panel_tile) applied to the n trailing
// columns X[:, pw .. pw + n); the tile's top pw rows go to `up` (row tile * pw), the rest to
// `down` (row down0 + tile * (256 - pw)).  ld, ldu and ldd are multiples of 4.
qrkit_status tsqr_panel_apply(qrkit_ctx* ctx, const float* X, int64_t ld, int64_t M, int pw, const float* T,
                              int n, float* up, int64_t ldu, float* down, int64_t ldd, int64_t down0,
                              int64_t tiles);
constexpr int kPanelCols = 32;    // column panel width of a (float) dense reduced block wider than that
constexpr int kMaxDenseS = 512;   // widest dense reduced block (float, column panels)
qrkit_status reduced_rhs_sort(qrkit_ctx* ctx, const int64_t* spos, const void* rhs, void* rhs_s, int64_t rows);
void release_band(Band& B);
qrkit_status launch_block_solve(qrkit_ctx* ctx, const void* J, const void* b, const void* D,
                                void* p, void* qtb, int refine_steps);
// Warp tasks of an uncoupled block plan: build (supertile of consecutive blocks, warps per
// CTA, task order: supertile-major, or key-major so that concurrent warps run one shape) and
// launch (factor + Q^T b + solve, then refinement of the selected blocks).
constexpr int64_t kDefaultSupertile = 65536;
qrkit_status build_block_tasks(qrkit_ctx* ctx, int64_t supertile, int warps, bool key_major);
qrkit_status launch_block_tasks(qrkit_ctx* ctx, const void* J, const void* b, void* p, void* qtb,
                                int refine_steps);
// Moré's stage 2 (Sec. 5.2) for the stored block factor: p from [R_i; lambda^(1/2) D_i] and the
// top m_i entries of qtb per block (D null: column norms of R_i).
qrkit_status more_stage2(qrkit_ctx* ctx, const void* qtb, const void* D, double lambda, void* p);
qrkit_status more_trust_region(qrkit_ctx* ctx, const void* qtb, const void* D, double delta, double sigma,
                               int max_iter, double* lambda, void* p, int* iterations);
// The warp-task factor (task planes) copied into J's packing and tau into column order.
qrkit_status unpack_block_tasks_factor(qrkit_ctx* ctx, void* factor_out, void* tau_out);
void release_block_tasks(Plan& P);

}  // namespace qrkit

#define QRKIT_CUDA_TRY(ctx, call)                                  \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ::qrkit::cuda_fail(ctx, e_, #call); \
  } while (0)
