// Context, structure plan and the C-ABI entry points.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace qrkit {

TileBudget block_solve_budget(size_t elem);
int block_solve_max_rows();
int block_solve_max_cols();

qrkit_status fail(qrkit_ctx* ctx, qrkit_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

qrkit_status cuda_fail(qrkit_ctx* ctx, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(ctx, e == cudaErrorMemoryAllocation ? QRKIT_ENOMEM : QRKIT_ECUDA, msg);
}

void release(DevBuf& buf) {
  if (buf.ptr) cudaFree(buf.ptr);
  buf.ptr = nullptr;
  buf.bytes = 0;
}

qrkit_status ensure(qrkit_ctx* ctx, DevBuf& buf, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  if (buf.ptr && buf.bytes >= bytes) return QRKIT_OK;
  release(buf);
  cudaError_t e = cudaMalloc(&buf.ptr, bytes);
  if (e != cudaSuccess) {
    buf.ptr = nullptr;
    return cuda_fail(ctx, e, what);
  }
  buf.bytes = bytes;
  return QRKIT_OK;
}

static qrkit_status upload(qrkit_ctx* ctx, DevBuf& buf, const void* host, size_t bytes,
                           const char* what) {
  qrkit_status st = ensure(ctx, buf, bytes, what);
  if (st != QRKIT_OK) return st;
  if (bytes) QRKIT_CUDA_TRY(ctx, cudaMemcpy(buf.ptr, host, bytes, cudaMemcpyHostToDevice));
  return QRKIT_OK;
}

static void release_plan(Plan& P) {
  release_block_tasks(P);
  release(P.d_val_off);
  release(P.d_row_off);
  release(P.d_col_off);
  release(P.d_start);
  release(P.d_seg);
  release(P.d_n);
  release(P.d_m);
  release(P.d_tile_block);
  release(P.d_tile_val);
  release(P.d_tile_row);
  release(P.d_tile_col);
  P = Plan();
}

// Greedy tile schedule: consecutive blocks while every budget holds.
void cut_tiles_for(Plan& P) {
  const TileBudget& B = P.budget;
  P.tile_block.assign(1, 0);
  P.tile_val.assign(1, 0);
  P.tile_row.assign(1, 0);
  P.tile_col.assign(1, 0);
  int64_t nb = 0, nv = 0, nr = 0, nc = 0, np = 0;
  int64_t val = 0, row = 0, col = 0;
  for (int64_t i = 0; i < P.K; ++i) {
    const int64_t n = P.n[i], m = P.m[i];
    const int64_t pad = 4 * ((n + 3) / 4) * m;   // rows padded to a multiple of 4
    if (nb > 0 && (nb + 1 > B.blocks || nv + n * m > B.values || nr + n > B.rows ||
                   nc + m > B.cols || np + pad > B.padded)) {
      P.tile_block.push_back(i);
      P.tile_val.push_back(val);
      P.tile_row.push_back(row);
      P.tile_col.push_back(col);
      nb = nv = nr = nc = np = 0;
    }
    nb += 1; nv += n * m; nr += n; nc += m; np += pad;
    val += n * m; row += n; col += m;
  }
  P.tile_block.push_back(P.K);
  P.tile_val.push_back(val);
  P.tile_row.push_back(row);
  P.tile_col.push_back(col);
  P.num_tiles = (int64_t)P.tile_block.size() - 1;
}

static qrkit_status plan_blocks(qrkit_ctx* ctx, const qrkit_structure* s) {
  Plan& P = ctx->plan;
  if (s->num_blocks < 1) return fail(ctx, QRKIT_EINVAL, "num_blocks must be >= 1");
  if (!s->block_rows || !s->block_cols)
    return fail(ctx, QRKIT_EINVAL, "block_rows and block_cols are required");
  if (s->coupled_kind < QRKIT_COUPLED_NONE || s->coupled_kind > QRKIT_COUPLED_WINDOW)
    return fail(ctx, QRKIT_EINVAL, "unknown coupled_kind");
  if (s->coupled_kind != QRKIT_COUPLED_NONE && s->shared_cols < 1)
    return fail(ctx, QRKIT_EINVAL, "shared_cols must be >= 1 for a coupled structure");
  if (s->coupled_kind == QRKIT_COUPLED_WINDOW) {
    if (s->window < 1 || s->window > s->shared_cols)
      return fail(ctx, QRKIT_EINVAL, "window must be in [1, shared_cols]");
    if (!s->window_start) return fail(ctx, QRKIT_EINVAL, "window_start is required");
  }
  P.K = s->num_blocks;
  P.n.assign(s->block_rows, s->block_rows + P.K);
  P.m.assign(s->block_cols, s->block_cols + P.K);
  const int maxr = block_solve_max_rows(), maxc = block_solve_max_cols();
  for (int64_t i = 0; i < P.K; ++i) {
    const int n = P.n[i], m = P.m[i];
    if (n < 1 || m < 1)
      return fail(ctx, QRKIT_EINVAL, "block " + std::to_string(i) + ": empty block");
    if (n > maxr || m > maxc)
      return fail(ctx, QRKIT_EUNSUPPORTED,
                  "block " + std::to_string(i) + ": " + std::to_string(n) + "x" +
                      std::to_string(m) + " exceeds the block kernel's 16 rows x 8 columns");
    P.rows += n;
    P.cols += m;
    P.values += (int64_t)n * m;
    P.max_n = std::max(P.max_n, n);
    P.max_m = std::max(P.max_m, m);
    if (n < m && P.first_wide < 0) P.first_wide = i;
    if (n + m > 16 && P.first_tall_aug < 0) P.first_tall_aug = i;
  }
  P.val_off.assign(P.K + 1, 0);
  P.row_off.assign(P.K + 1, 0);
  P.col_off.assign(P.K + 1, 0);
  for (int64_t i = 0; i < P.K; ++i) {
    P.val_off[i + 1] = P.val_off[i] + (int64_t)P.n[i] * P.m[i];
    P.row_off[i + 1] = P.row_off[i] + P.n[i];
    P.col_off[i + 1] = P.col_off[i] + P.m[i];
  }
  if (s->coupled_kind == QRKIT_COUPLED_WINDOW) {
    // segments of S (Sec. 4.2 horizontal concatenation of independent banded parts)
    const int64_t nseg = s->num_segments > 0 ? s->num_segments : 1;
    if (s->num_segments > 1 && (!s->segment_cols || !s->segment_blocks))
      return fail(ctx, QRKIT_EINVAL, "segment_cols and segment_blocks are required for num_segments > 1");
    if (s->num_segments == 1 && s->segment_cols && s->segment_blocks) {
      P.seg_cols.assign(1, s->segment_cols[0]);
      P.seg_blocks.assign(1, s->segment_blocks[0]);
    } else if (s->num_segments > 1) {
      P.seg_cols.assign(s->segment_cols, s->segment_cols + nseg);
      P.seg_blocks.assign(s->segment_blocks, s->segment_blocks + nseg);
    } else {
      P.seg_cols.assign(1, s->shared_cols);
      P.seg_blocks.assign(1, P.K);
    }
    P.seg_col0.assign(nseg + 1, 0);
    P.seg_blk0.assign(nseg + 1, 0);
    for (int64_t k = 0; k < nseg; ++k) {
      if (P.seg_cols[k] < 1 || P.seg_blocks[k] < 0)
        return fail(ctx, QRKIT_EINVAL, "segment " + std::to_string(k) + " is empty or negative");
      P.seg_col0[k + 1] = P.seg_col0[k] + P.seg_cols[k];
      P.seg_blk0[k + 1] = P.seg_blk0[k] + P.seg_blocks[k];
    }
    if (P.seg_col0[nseg] != s->shared_cols)
      return fail(ctx, QRKIT_EINVAL, "segment_cols must sum to shared_cols");
    if (P.seg_blk0[nseg] != P.K) return fail(ctx, QRKIT_EINVAL, "segment_blocks must sum to num_blocks");
    P.start.assign(s->window_start, s->window_start + P.K);
    for (int64_t k = 0; k < nseg; ++k)
      for (int64_t i = P.seg_blk0[k]; i < P.seg_blk0[k + 1]; ++i)
        if (P.start[i] < P.seg_col0[k] || P.start[i] >= P.seg_col0[k + 1])
          return fail(ctx, QRKIT_EINVAL, "window_start of block " + std::to_string(i) +
                                             " is outside its segment");
  }
  P.composed = s->coupled_kind != QRKIT_COUPLED_NONE;
  P.budget = block_solve_budget(elem_size(ctx));
  cut_tiles_for(P);
  qrkit_status st;
  if (!P.composed) {
    // the fused solve's default mapping: shape-uniform warp tasks
    P.mapping = 0;
    if ((st = build_block_tasks(ctx, kDefaultSupertile, 8, false)) != QRKIT_OK) return st;
  }
  {
    const size_t ob = (size_t)(P.K + 1) * sizeof(int64_t);
    if ((st = upload(ctx, P.d_val_off, P.val_off.data(), ob, "plan offsets")) != QRKIT_OK) return st;
    if ((st = upload(ctx, P.d_row_off, P.row_off.data(), ob, "plan offsets")) != QRKIT_OK) return st;
    if ((st = upload(ctx, P.d_col_off, P.col_off.data(), ob, "plan offsets")) != QRKIT_OK) return st;
    if (!P.start.empty()) {
      if ((st = upload(ctx, P.d_start, P.start.data(), P.K * sizeof(int32_t), "plan starts")) != QRKIT_OK)
        return st;
      std::vector<int64_t> seg(P.seg_blk0);
      seg.insert(seg.end(), P.seg_col0.begin(), P.seg_col0.end());
      if ((st = upload(ctx, P.d_seg, seg.data(), seg.size() * sizeof(int64_t), "plan segments")) != QRKIT_OK)
        return st;
    }
  }
  if ((st = upload(ctx, P.d_n, P.n.data(), P.K, "plan n")) != QRKIT_OK) return st;
  if ((st = upload(ctx, P.d_m, P.m.data(), P.K, "plan m")) != QRKIT_OK) return st;
  const size_t tb = (size_t)(P.num_tiles + 1) * sizeof(int64_t);
  if ((st = upload(ctx, P.d_tile_block, P.tile_block.data(), tb, "plan tiles")) != QRKIT_OK) return st;
  if ((st = upload(ctx, P.d_tile_val, P.tile_val.data(), tb, "plan tiles")) != QRKIT_OK) return st;
  if ((st = upload(ctx, P.d_tile_row, P.tile_row.data(), tb, "plan tiles")) != QRKIT_OK) return st;
  if ((st = upload(ctx, P.d_tile_col, P.tile_col.data(), tb, "plan tiles")) != QRKIT_OK) return st;
  const size_t es = elem_size(ctx);
  if ((st = ensure(ctx, ctx->ws.factor, (size_t)P.values * es, "factor workspace")) != QRKIT_OK)
    return st;
  if ((st = ensure(ctx, ctx->ws.tau, (size_t)P.cols * es, "tau workspace")) != QRKIT_OK) return st;
  P.s = *s;
  P.s.block_rows = nullptr;
  P.s.block_cols = nullptr;
  P.s.window_start = nullptr;
  P.s.segment_cols = nullptr;
  P.s.segment_blocks = nullptr;
  P.valid = true;
  return QRKIT_OK;
}

}  // namespace qrkit

using namespace qrkit;

extern "C" {

const char* qrkit_status_string(int st) {
  switch (st) {
    case QRKIT_OK: return "QRKIT_OK";
    case QRKIT_EINVAL: return "QRKIT_EINVAL";
    case QRKIT_ENOMEM: return "QRKIT_ENOMEM";
    case QRKIT_ECUDA: return "QRKIT_ECUDA";
    case QRKIT_ESINGULAR: return "QRKIT_ESINGULAR";
    case QRKIT_ENONFINITE: return "QRKIT_ENONFINITE";
    case QRKIT_ETIMEOUT: return "QRKIT_ETIMEOUT";
    case QRKIT_ENOTCONV: return "QRKIT_ENOTCONV";
    case QRKIT_EUNSUPPORTED: return "QRKIT_EUNSUPPORTED";
    case QRKIT_ESTATE: return "QRKIT_ESTATE";
    default: return "QRKIT_UNKNOWN";
  }
}

qrkit_status qrkit_create(qrkit_ctx** out, int device, void* stream, int precision) {
  if (!out) return QRKIT_EINVAL;
  *out = nullptr;
  if (precision < QRKIT_FP64 || precision > QRKIT_FP32) return QRKIT_EINVAL;
  qrkit_ctx* ctx = new (std::nothrow) qrkit_ctx();
  if (!ctx) return QRKIT_ENOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  ctx->precision = precision;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  ctx->max_smem_optin = (size_t)optin;
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? QRKIT_ENOMEM : QRKIT_ECUDA;
  }
  *out = ctx;
  return QRKIT_OK;
}

void qrkit_destroy(qrkit_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  release_lm(ctx->lm);
  release_mlp(ctx->mlp);
  release_plan(ctx->plan);
  release_composed(ctx->comp);
  release_band(ctx->band);
  release(ctx->ws.factor);
  release(ctx->ws.tau);
  release(ctx->ws.rlist);
  release(ctx->ws.rcount);
  release(ctx->ws.tlist);
  release(ctx->ws.tcount);
  release(ctx->more_sums);
  release(ctx->ws.tfactor);
  release(ctx->ws.ttau);
  release(ctx->ws.rrec);
  release(ctx->ws.qtb);
  if (ctx->d_status) cudaFree(ctx->d_status);
  delete ctx;
}

const char* qrkit_last_error(const qrkit_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "null context";
}

qrkit_status qrkit_plan(qrkit_ctx* ctx, const qrkit_structure* s) {
  if (!ctx) return QRKIT_EINVAL;
  if (!s) return fail(ctx, QRKIT_EINVAL, "null structure");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  release_plan(ctx->plan);
  release_composed(ctx->comp);
  release_band(ctx->band);
  release_lm(ctx->lm);
  ctx->factored = false;
  if (s->kind == QRKIT_STRUCT_BLOCKS) return plan_blocks(ctx, s);
  if (s->kind == QRKIT_STRUCT_BANDED) return banded_plan(ctx, s);
  return fail(ctx, QRKIT_EINVAL, "unknown structure kind");
}

qrkit_status qrkit_factor_solve(qrkit_ctx* ctx, const void* J, const void* b, const void* D,
                                double lambda, void* p, void* qtb, int refine_steps) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->plan.valid) return fail(ctx, QRKIT_ESTATE, "qrkit_factor_solve before qrkit_plan");
  const Plan& P = ctx->plan;
  if (P.s.kind == QRKIT_STRUCT_BANDED) {
    if (!J || !b || !p) return fail(ctx, QRKIT_EINVAL, "J, b and p are required");
    if (qtb) return fail(ctx, QRKIT_EINVAL, "qtb is not available for banded structures");
    if (!(lambda >= 0.0)) return fail(ctx, QRKIT_EINVAL, "lambda must be >= 0");
    if (refine_steps < 0 || refine_steps > 8) return fail(ctx, QRKIT_EINVAL, "refine_steps must be in [0, 8]");
    QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    qrkit_status st = banded_factor_solve(ctx, J, b, D, lambda, p, refine_steps);
    if (st == QRKIT_OK) ctx->band_factored = true;
    return st;
  }
  if (P.s.kind != QRKIT_STRUCT_BLOCKS || P.s.coupled_kind != QRKIT_COUPLED_NONE)
    return fail(ctx, QRKIT_EINVAL, "qrkit_factor_solve needs a block-diagonal or banded structure");
  ctx->comp_factored = false;
  if (!J || !b || !p) return fail(ctx, QRKIT_EINVAL, "J, b and p are required");
  if (!(lambda >= 0.0)) return fail(ctx, QRKIT_EINVAL, "lambda must be >= 0");
  if (refine_steps < 0 || refine_steps > 8) return fail(ctx, QRKIT_EINVAL, "refine_steps must be in [0, 8]");
  if (P.first_wide >= 0)
    return fail(ctx, QRKIT_EINVAL, "block " + std::to_string(P.first_wide) + " has fewer rows than columns");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (lambda > 0.0) {
    // Moré's two factorizations (Sec. 5.2): the undamped fused QR (its Q^T b kept), then the
    // QR of [R_i; lambda^(1/2) D_i] per block; no refinement on this path
    void* q = qtb;
    if (!q) {
      qrkit_status r = ensure(ctx, ctx->ws.qtb, (size_t)P.rows * elem_size(ctx), "damped solve Q^T b");
      if (r != QRKIT_OK) return r;
      q = ctx->ws.qtb.ptr;
    }
    qrkit_status st = launch_block_solve(ctx, J, b, nullptr, p, q, 0);
    if (st != QRKIT_OK) return st;
    ctx->factored = true;
    ctx->factor_in_planes = ctx->plan.mapping == 0 && ctx->plan.num_tasks > 0;
    return more_stage2(ctx, q, D, lambda, p);
  }
  qrkit_status st = launch_block_solve(ctx, J, b, D, p, qtb, refine_steps);
  if (st == QRKIT_OK) {
    ctx->factored = true;
    ctx->factor_in_planes = ctx->plan.mapping == 0 && ctx->plan.num_tasks > 0;
  }
  return st;
}

qrkit_status qrkit_more_solve(qrkit_ctx* ctx, const void* qtb, const void* D, double lambda, void* p) {
  if (!ctx) return QRKIT_EINVAL;
  const Plan& P = ctx->plan;
  if (!P.valid || P.s.kind != QRKIT_STRUCT_BLOCKS || P.s.coupled_kind != QRKIT_COUPLED_NONE)
    return fail(ctx, QRKIT_ESTATE, "qrkit_more_solve needs a block-diagonal plan");
  if (!ctx->factored) return fail(ctx, QRKIT_ESTATE, "qrkit_more_solve before qrkit_factor_solve");
  if (!qtb || !p) return fail(ctx, QRKIT_EINVAL, "qtb and p are required");
  if (!(lambda >= 0.0)) return fail(ctx, QRKIT_EINVAL, "lambda must be >= 0");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return more_stage2(ctx, qtb, D, lambda, p);
}

qrkit_status qrkit_more_trust_region(qrkit_ctx* ctx, const void* qtb, const void* D, double delta, double sigma,
                                     int max_iter, double* lambda, void* p, int* iterations) {
  if (!ctx) return QRKIT_EINVAL;
  const Plan& P = ctx->plan;
  if (!P.valid || P.s.kind != QRKIT_STRUCT_BLOCKS || P.s.coupled_kind != QRKIT_COUPLED_NONE)
    return fail(ctx, QRKIT_ESTATE, "qrkit_more_trust_region needs a block-diagonal plan");
  if (!ctx->factored) return fail(ctx, QRKIT_ESTATE, "qrkit_more_trust_region before qrkit_factor_solve");
  if (!qtb || !p || !lambda) return fail(ctx, QRKIT_EINVAL, "qtb, p and lambda are required");
  if (!(delta > 0.0) || !(sigma > 0.0 && sigma < 1.0) || max_iter < 1)
    return fail(ctx, QRKIT_EINVAL, "need delta > 0, 0 < sigma < 1, max_iter >= 1");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return more_trust_region(ctx, qtb, D, delta, sigma, max_iter, lambda, p, iterations);
}

static qrkit_status need_dense_plan(qrkit_ctx* ctx, const char* what) {
  const Plan& P = ctx->plan;
  if (!P.valid || P.s.kind != QRKIT_STRUCT_BLOCKS || P.s.coupled_kind != QRKIT_COUPLED_DENSE)
    return fail(ctx, QRKIT_ESTATE, std::string(what) + " needs a plan with a dense S");
  return QRKIT_OK;
}

qrkit_status qrkit_column_sumsq(qrkit_ctx* ctx, const void* J, const void* S, double* sq) {
  if (!ctx) return QRKIT_EINVAL;
  const Plan& P = ctx->plan;
  if (!P.valid || P.s.kind != QRKIT_STRUCT_BLOCKS) return fail(ctx, QRKIT_ESTATE, "qrkit_column_sumsq needs a block plan");
  if (!J || !sq || (P.s.coupled_kind != QRKIT_COUPLED_NONE && !S)) return fail(ctx, QRKIT_EINVAL, "J, S and sq are required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return composed_column_sumsq(ctx, J, S, sq);
}

qrkit_status qrkit_norms_from_sumsq(qrkit_ctx* ctx, const double* sq, int64_t n, void* D) {
  if (!ctx) return QRKIT_EINVAL;
  if (!sq || !D || n < 1) return fail(ctx, QRKIT_EINVAL, "sq, D and n >= 1 are required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return composed_norms_from_sumsq(ctx, sq, n, D);
}

qrkit_status qrkit_get_reduced_r(qrkit_ctx* ctx, void* R) {
  if (!ctx) return QRKIT_EINVAL;
  qrkit_status st = need_dense_plan(ctx, "qrkit_get_reduced_r");
  if (st != QRKIT_OK) return st;
  if (!ctx->comp_factored) return fail(ctx, QRKIT_ESTATE, "qrkit_get_reduced_r before qrkit_factor");
  if (!R) return fail(ctx, QRKIT_EINVAL, "R is required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return composed_reduced_r(ctx, R);
}

qrkit_status qrkit_solve_blocks(qrkit_ctx* ctx, const void* qtb, void* p) {
  if (!ctx) return QRKIT_EINVAL;
  const Plan& P = ctx->plan;
  if (!P.valid || P.s.kind != QRKIT_STRUCT_BLOCKS || P.s.coupled_kind == QRKIT_COUPLED_WINDOW)
    return fail(ctx, QRKIT_ESTATE, "qrkit_solve_blocks needs a block plan without windows");
  if (!ctx->comp_factored) return fail(ctx, QRKIT_ESTATE, "qrkit_solve_blocks before qrkit_factor");
  if (!qtb || !p) return fail(ctx, QRKIT_EINVAL, "qtb and p are required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return composed_solve_blocks(ctx, qtb, p);
}

qrkit_status qrkit_set_wait_limit(qrkit_ctx* ctx, int64_t polls) {
  if (!ctx) return QRKIT_EINVAL;
  if (polls < 0) return fail(ctx, QRKIT_EINVAL, "polls must be >= 0");
  ctx->wait_limit = polls;
  return QRKIT_OK;
}

qrkit_status qrkit_set_refinement(qrkit_ctx* ctx, double select, int residual) {
  if (!ctx) return QRKIT_EINVAL;
  if (!(select >= 0.0 && select <= 1.0)) return fail(ctx, QRKIT_EINVAL, "select must be in [0, 1]");
  if (residual != QRKIT_RESIDUAL_DOT2 && residual != QRKIT_RESIDUAL_FP64)
    return fail(ctx, QRKIT_EINVAL, "residual must be QRKIT_RESIDUAL_DOT2 or QRKIT_RESIDUAL_FP64");
  ctx->refine_select = (float)select;
  ctx->refine_residual = residual;
  return QRKIT_OK;
}

qrkit_status qrkit_factor(qrkit_ctx* ctx, const void* J, const void* S, const void* D, double lambda) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->plan.valid) return fail(ctx, QRKIT_ESTATE, "qrkit_factor before qrkit_plan");
  const Plan& P = ctx->plan;
  if (P.s.kind != QRKIT_STRUCT_BLOCKS)
    return fail(ctx, QRKIT_EUNSUPPORTED, "qrkit_factor: only block structures in this build");
  if (!J) return fail(ctx, QRKIT_EINVAL, "J is required");
  if (P.s.coupled_kind != QRKIT_COUPLED_NONE && !S)
    return fail(ctx, QRKIT_EINVAL, "S is required for a coupled structure");
  if (!(lambda >= 0.0)) return fail(ctx, QRKIT_EINVAL, "lambda must be >= 0");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  ctx->comp_factored = false;
  qrkit_status st = composed_factor(ctx, J, S, D, lambda);
  if (st != QRKIT_OK) return st;
  ctx->comp.J = J;
  ctx->comp.S = S;
  ctx->comp_factored = true;
  return QRKIT_OK;
}

qrkit_status qrkit_apply_qt(qrkit_ctx* ctx, const void* b, void* qtb) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->comp_factored) return fail(ctx, QRKIT_ESTATE, "qrkit_apply_qt before qrkit_factor");
  if (!b || !qtb) return fail(ctx, QRKIT_EINVAL, "b and qtb are required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return composed_apply_qt(ctx, b, qtb);
}

qrkit_status qrkit_solve_r(qrkit_ctx* ctx, const void* qtb, void* p) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->comp_factored) return fail(ctx, QRKIT_ESTATE, "qrkit_solve_r before qrkit_factor");
  if (!qtb || !p) return fail(ctx, QRKIT_EINVAL, "qtb and p are required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return composed_solve_r(ctx, qtb, p);
}

qrkit_status qrkit_solve(qrkit_ctx* ctx, const void* b, void* p, int refine_steps) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->comp_factored) return fail(ctx, QRKIT_ESTATE, "qrkit_solve before qrkit_factor");
  if (!b || !p) return fail(ctx, QRKIT_EINVAL, "b and p are required");
  if (refine_steps < 0 || refine_steps > 8) return fail(ctx, QRKIT_EINVAL, "refine_steps must be in [0, 8]");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return composed_solve(ctx, ctx->comp.J, ctx->comp.S, b, p, refine_steps);
}

qrkit_status qrkit_get_band_factor(qrkit_ctx* ctx, void* Rw, void* c, double* res2) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->band_factored) return fail(ctx, QRKIT_ESTATE, "no banded factor stored");
  qrkit_status st = banded_get_factor(ctx, Rw, c, res2);
  if (st != QRKIT_OK) return st;
  QRKIT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return QRKIT_OK;
}

qrkit_status qrkit_get_factor(qrkit_ctx* ctx, void* factor_out, void* tau_out) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->factored) return fail(ctx, QRKIT_ESTATE, "no factor stored");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (ctx->factor_in_planes) return unpack_block_tasks_factor(ctx, factor_out, tau_out);
  const size_t es = elem_size(ctx);
  if (factor_out)
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(factor_out, ctx->ws.factor.ptr, (size_t)ctx->plan.values * es,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
  if (tau_out)
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(tau_out, ctx->ws.tau.ptr, (size_t)ctx->plan.cols * es,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
  return QRKIT_OK;
}

qrkit_status qrkit_set_window_start(qrkit_ctx* ctx, const int32_t* start) {
  if (!ctx) return QRKIT_EINVAL;
  const Plan& P = ctx->plan;
  if (!P.valid || P.s.kind != QRKIT_STRUCT_BLOCKS || P.s.coupled_kind != QRKIT_COUPLED_WINDOW)
    return fail(ctx, QRKIT_ESTATE, "qrkit_set_window_start needs a windowed block plan");
  if (!start) return fail(ctx, QRKIT_EINVAL, "start is required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  ctx->comp_factored = false;
  return window_start_copy(ctx, start);
}

qrkit_status qrkit_get_row_order(qrkit_ctx* ctx, int64_t* order) {
  if (!ctx) return QRKIT_EINVAL;
  const Plan& P = ctx->plan;
  if (!P.valid || P.s.kind != QRKIT_STRUCT_BLOCKS || P.s.coupled_kind != QRKIT_COUPLED_WINDOW)
    return fail(ctx, QRKIT_ESTATE, "qrkit_get_row_order needs a windowed block plan");
  if (!ctx->comp_factored) return fail(ctx, QRKIT_ESTATE, "qrkit_get_row_order before qrkit_factor");
  if (!order) return fail(ctx, QRKIT_EINVAL, "order is required");
  if (ctx->comp.red_rows > 0)
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(order, ctx->comp.order.ptr, (size_t)ctx->comp.red_rows * sizeof(int64_t),
                                        cudaMemcpyDeviceToDevice, ctx->stream));
  return QRKIT_OK;
}

qrkit_status qrkit_sync_status(qrkit_ctx* ctx) {
  if (!ctx) return QRKIT_EINVAL;
  QRKIT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  int h = 0;
  QRKIT_CUDA_TRY(ctx, cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  QRKIT_CUDA_TRY(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  if (h != 0) return fail(ctx, (qrkit_status)h, std::string("device reported ") + qrkit_status_string(h));
  return QRKIT_OK;
}

int64_t qrkit_launch_count(const qrkit_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
