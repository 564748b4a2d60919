// Levenberg-Marquardt iterations on the device (Sec. 2; "Backtrack LM" of Sec. 5.2): every
// iteration factors P_r [J; lambda^(1/2) D] once by the composed QR and takes or rejects the
// step by the gain ratio, with Nielsen's damping update.
//
// Model: 2-D points on an open uniform cubic B-spline, one latent parameter t_i per point and
// the control points shared (the block-angular shape of the paper's surface-fitting problems,
// Sec. 6.2 / Fig. 5a): J = [blkdiag(2x1 blocks) | S], each point's two rows touching 8
// consecutive shared columns (a window, Sec. 4.2 + Sec. 4.4).  Several independent problems
// are solved together: their shared columns are separate segments of S, every problem has
// its own lambda, nu and acceptance.
//
//   x = [t of all points | control points of problem 0 (x0, y0, x1, y1, ..), problem 1, ..]
//   seg = clamp(floor(t), 0, Kc - 4), u = t - seg, curve(t) = sum_q B_q(u) P_{seg+q}
//   f_i = curve(t_i) - data_i, cost = 1/2 ||f||^2, b = -f
//   D = column norms of J (zero -> 1); the damping enters as E = lambda_k^(1/2) D per column
//   pred = 1/2 p^T (lambda D^2 p + J^T b) = 1/2 (sum_j E_j^2 p_j^2 + (J p)^T b)
//   rho = (cost(x) - cost(x + p)) / pred (-1 when pred <= 0)
//   Nielsen: rho > 0 -> accept, lambda *= max(1/3, 1 - (2 rho - 1)^3), nu = 2;
//            else lambda *= nu, nu *= 2
// x, the data, residuals and all costs are double; J, S and b are rounded once to the
// context's precision for the factorization.  The state of every problem stays on the device
// between the kernels of an iteration, so an iteration is a fixed sequence of launches and
// can be captured into a CUDA graph (qrkit_lm_run).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"
#include "mlp_policy.cuh"

namespace qrkit {

constexpr int kTilePts = 256;   // points per reduction tile (tiles never cross problems)
constexpr int kEvalSumCols = 2048;   // problems up to this many columns: S column sums per tile in shared memory

struct LMTables {
  int64_t B = 0, NP = 0, s = 0, N = 0, num_tiles = 0;
  const int64_t* p0 = nullptr;         // B + 1: first point of problem k
  const int64_t* c0 = nullptr;         // B + 1: first shared column of problem k (within S)
  const int64_t* tile_p0 = nullptr;    // num_tiles + 1
  const int32_t* tile_prob = nullptr;  // num_tiles
  const int64_t* prob_tile0 = nullptr; // B + 1
  const int32_t* col_prob = nullptr;   // N: problem of each column
};

struct LM {
  LMTables t;
  std::vector<int64_t> h_p0, h_c0, h_tile_p0, h_prob_tile0;
  DevBuf tabs, tile_prob, col_prob;
  const double* data = nullptr;        // caller's points (device)
  DevBuf J, S, b, p, start, d2, E, xnew, tile_cost, tile_new, tile_pred, state, ndone;
  DevBuf hist, feat;                   // per problem: step history (12) and policy features (16)
  bool policy = false;                 // damping from the MLP after accepted steps
  bool prepared = false;
  int sum_cols = 0;                    // columns of the widest problem when it fits a tile's shared sums
  cudaGraphExec_t graph = nullptr;
  int graph_refine = -1;
  int64_t graph_launches = 0;          // kernels in one captured iteration
  double graph_ftol = 0.0;
  const double* graph_x = nullptr;
};

void release_lm(LM*& lm) {
  if (!lm) return;
  if (lm->graph) cudaGraphExecDestroy(lm->graph);
  for (DevBuf* b : {&lm->tabs, &lm->tile_prob, &lm->col_prob, &lm->J, &lm->S, &lm->b, &lm->p, &lm->start,
                    &lm->d2, &lm->E, &lm->xnew, &lm->tile_cost, &lm->tile_new, &lm->tile_pred, &lm->state,
                    &lm->ndone, &lm->hist, &lm->feat})
    release(*b);
  delete lm;
  lm = nullptr;
}

namespace {

// Uniform cubic B-spline basis and its derivative at u in [0, 1] (extrapolated outside),
// in Horner form with multiplications only (double division is slow on this part):
//   6 B_0 = (1-u)^3, 6 B_1 = (3u - 6) u^2 + 4, 6 B_2 = ((-3u + 3) u + 3) u + 1, 6 B_3 = u^3,
//   B_0' = -(1-u)^2 / 2, B_1' = (3u/2 - 2) u, B_2' = (-3u/2 + 1) u + 1/2, B_3' = u^2 / 2.
__device__ __forceinline__ void bspline(double u, double B[4], double dB[4]) {
  const double sixth = 1.0 / 6.0;
  const double v = 1.0 - u, u2 = u * u;
  B[0] = v * v * v * sixth;
  B[1] = fma(fma(3.0, u, -6.0), u2, 4.0) * sixth;
  B[2] = fma(fma(fma(-3.0, u, 3.0), u, 3.0), u, 1.0) * sixth;
  B[3] = u2 * u * sixth;
  dB[0] = -0.5 * v * v;
  dB[1] = fma(1.5, u, -2.0) * u;
  dB[2] = fma(fma(-1.5, u, 1.0), u, 0.5);
  dB[3] = 0.5 * u2;
}

// The basis alone (the trial cost needs no derivative).
__device__ __forceinline__ void bspline_values(double u, double B[4]) {
  const double sixth = 1.0 / 6.0;
  const double v = 1.0 - u, u2 = u * u;
  B[0] = v * v * v * sixth;
  B[1] = fma(fma(3.0, u, -6.0), u2, 4.0) * sixth;
  B[2] = fma(fma(fma(-3.0, u, 3.0), u, 3.0), u, 1.0) * sixth;
  B[3] = u2 * u * sixth;
}

__device__ __forceinline__ int64_t segment_of(double t, int64_t Kc) {
  const double hi = (double)(Kc - 4);
  double f = floor(t);
  if (!(f >= 0.0)) f = 0.0;   // also NaN
  if (f > hi) f = hi;
  return (int64_t)f;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;   // valid in thread 0
}

// Residual, Jacobian blocks, windows, b = -f, squared column norms and the cost per tile.
// A tile lies in one problem: when the problem's columns fit (sum_cols > 0), the squared
// column sums of S are gathered in shared memory and leave the tile with one global atomic per
// column touched, instead of eight per point.
template <typename T>
__global__ void __launch_bounds__(kTilePts)
cf_eval_kernel(LMTables t, const double* x, const double* data, T* J, T* S, T* b, int32_t* start,
               double* d2, double* tile_cost, int sum_cols) {
  __shared__ double red[kTilePts / 32];
  extern __shared__ double scol[];
  const int64_t tile = blockIdx.x;
  const int64_t i = t.tile_p0[tile] + threadIdx.x;
  const int kt = t.tile_prob[tile];
  const int ncol = (int)(t.c0[kt + 1] - t.c0[kt]);
  const bool tile_sum = ncol <= sum_cols;
  if (tile_sum) {
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) scol[c] = 0.0;
    __syncthreads();
  }
  double fsq = 0.0;
  if (i < t.tile_p0[tile + 1]) {
    const int k = kt;
    const int64_t Kc = (t.c0[k + 1] - t.c0[k]) / 2;
    const double ti = x[i];
    const int64_t seg = segment_of(ti, Kc);
    double Bv[4], dB[4];
    bspline(ti - (double)seg, Bv, dB);
    const double* P = x + t.NP + t.c0[k] + 2 * seg;
    double cx = 0, cy = 0, dx = 0, dy = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      cx += Bv[q] * P[2 * q];
      cy += Bv[q] * P[2 * q + 1];
      dx += dB[q] * P[2 * q];
      dy += dB[q] * P[2 * q + 1];
    }
    const double fx = cx - data[2 * i], fy = cy - data[2 * i + 1];
    fsq = fx * fx + fy * fy;
    const T jx = (T)dx, jy = (T)dy;
    J[2 * i] = jx;
    J[2 * i + 1] = jy;
    b[2 * i] = (T)(-fx);
    b[2 * i + 1] = (T)(-fy);
    d2[i] = (double)jx * (double)jx + (double)jy * (double)jy;
    T* Si = S + 16 * i;   // 2 x 8, column-major
    const int64_t col = t.c0[k] + 2 * seg;
    start[i] = (int32_t)col;
    double* dS = d2 + t.NP + col;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T v = (T)Bv[q];
      Si[4 * q + 0] = v;      // (row x, column 2q)
      Si[4 * q + 1] = T(0);   // (row y, column 2q)
      Si[4 * q + 2] = T(0);   // (row x, column 2q + 1)
      Si[4 * q + 3] = v;      // (row y, column 2q + 1)
      const double v2 = (double)v * (double)v;
      if (v2 != 0.0) {
        if (tile_sum) {
          atomicAdd(&scol[2 * seg + 2 * q], v2);
          atomicAdd(&scol[2 * seg + 2 * q + 1], v2);
        } else {
          atomicAdd(dS + 2 * q, v2);
          atomicAdd(dS + 2 * q + 1, v2);
        }
      }
    }
  }
  const double s = block_sum(fsq, red);
  if (threadIdx.x == 0) tile_cost[tile] = s;
  if (tile_sum) {
    __syncthreads();
    double* dP = d2 + t.NP + t.c0[kt];
    for (int c = threadIdx.x; c < ncol; c += blockDim.x)
      if (scol[c] != 0.0) atomicAdd(dP + c, scol[c]);
  }
}

// E_j = lambda_k^(1/2) D_j with D_j = ||column j of J|| (zero -> 1).
__global__ void lm_damp_kernel(LMTables t, const double* d2, const qrkit_lm_state* st, double* E) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= t.N) return;
  double d = sqrt(d2[j]);
  if (d == 0.0) d = 1.0;
  E[j] = sqrt(st[t.col_prob[j]].lambda) * d;
}

// f = curve(t) - data per point (two values), double.
__global__ void cf_residual_kernel(LMTables t, const double* x, const double* data, double* f) {
  const int64_t tile = blockIdx.x;
  const int64_t i = t.tile_p0[tile] + threadIdx.x;
  if (i >= t.tile_p0[tile + 1]) return;
  const int k = t.tile_prob[tile];
  const int64_t Kc = (t.c0[k + 1] - t.c0[k]) / 2;
  const double ti = x[i];
  const int64_t seg = segment_of(ti, Kc);
  double Bv[4], dB[4];
  bspline(ti - (double)seg, Bv, dB);
  const double* P = x + t.NP + t.c0[k] + 2 * seg;
  double cx = 0, cy = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    cx += Bv[q] * P[2 * q];
    cy += Bv[q] * P[2 * q + 1];
  }
  f[2 * i] = cx - data[2 * i];
  f[2 * i + 1] = cy - data[2 * i + 1];
}

template <typename T>
__global__ void lm_xnew_kernel(int64_t N, const double* x, const T* p, double* xnew) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) xnew[j] = x[j] + (double)p[j];
}

// Cost at x + p and the row part of the predicted decrease, (J p)^T b + E_t^2 p_t^2, per tile.
template <typename T>
__global__ void __launch_bounds__(kTilePts)
cf_trial_kernel(LMTables t, const double* xnew, const double* data, const T* J, const T* S, const T* b,
                const T* p, const double* E, const int32_t* start, double* tile_new, double* tile_pred) {
  __shared__ double red[kTilePts / 32];
  const int64_t tile = blockIdx.x;
  const int64_t i = t.tile_p0[tile] + threadIdx.x;
  double fsq = 0.0, pr = 0.0;
  if (i < t.tile_p0[tile + 1]) {
    const int k = t.tile_prob[tile];
    const int64_t Kc = (t.c0[k + 1] - t.c0[k]) / 2;
    const double ti = xnew[i];
    const int64_t seg = segment_of(ti, Kc);
    double Bv[4];
    bspline_values(ti - (double)seg, Bv);
    const double* P = xnew + t.NP + t.c0[k] + 2 * seg;
    double cx = 0, cy = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      cx += Bv[q] * P[2 * q];
      cy += Bv[q] * P[2 * q + 1];
    }
    const double fx = cx - data[2 * i], fy = cy - data[2 * i + 1];
    fsq = fx * fx + fy * fy;
    // (J p) at the linearisation point, with the system's own J, S and b; in the context
    // precision (a relative error of the order of its rounding in the predicted decrease moves
    // the gain ratio by as little, far below what the damping rule resolves)
    const T pt = p[i];
    T jx = J[2 * i] * pt, jy = J[2 * i + 1] * pt;
    const T* Si = S + 16 * i;
    const T* pS = p + t.NP + start[i];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      jx += Si[2 * c] * pS[c];
      jy += Si[2 * c + 1] * pS[c];
    }
    const T e = (T)E[i];
    pr = (double)(jx * b[2 * i] + jy * b[2 * i + 1] + e * e * pt * pt);
  }
  const double s1 = block_sum(fsq, red);
  __syncthreads();
  const double s2 = block_sum(pr, red);
  if (threadIdx.x == 0) {
    tile_new[tile] = s1;
    tile_pred[tile] = s2;
  }
}

constexpr int kHist = 12;   // rho, accepted, log cost ratio of the last 4 steps

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// One warp per problem: costs, predicted decrease, gain ratio, then the damping update:
// Nielsen's rule, or after an accepted step (when the policy is on) lambda * multiplier of the
// MLP's class for the features of the step history; stop rule.
template <typename T>
__global__ void lm_update_kernel(LMTables t, const double* tile_cost, const double* tile_new,
                                 const double* tile_pred, const double* E, const T* p, qrkit_lm_state* st,
                                 double ftol, int* ndone, MlpDev w, float* hist, float* feat) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= t.B) return;
  double c = 0, cn = 0, pr = 0;
  for (int64_t q = t.prob_tile0[k] + lane; q < t.prob_tile0[k + 1]; q += 32) {
    c += tile_cost[q];
    cn += tile_new[q];
    pr += tile_pred[q];
  }
  for (int64_t j = t.NP + t.c0[k] + lane; j < t.NP + t.c0[k + 1]; j += 32) {
    const double pj = (double)p[j];
    pr += E[j] * E[j] * pj * pj;
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, d);
    cn += __shfl_xor_sync(0xffffffffu, cn, d);
    pr += __shfl_xor_sync(0xffffffffu, pr, d);
  }
  qrkit_lm_state s = st[k];
  if (s.done) {
    if (lane == 0) {
      s.accepted = 0;
      st[k] = s;
      atomicAdd(ndone, 1);
    }
    return;
  }
  const double cost = 0.5 * c, cost_new = 0.5 * cn, pred = 0.5 * pr;
  const double rho = pred > 0.0 ? (cost - cost_new) / pred : -1.0;
  const bool acc = rho > 0.0;
  // step history and features (every lane computes the same values)
  float* hk = hist + k * kHist;
  float h[kHist];
#pragma unroll
  for (int q = 0; q < kHist; ++q) h[q] = s.iteration == 0 ? 0.f : hk[q];
  const float ratio = cost > 0.0 ? (float)log10(fmax(cost_new / cost, 1e-30)) : 0.f;
  const float pratio = cost > 0.0 ? (float)log10(fmax(pred / cost, 1e-30)) : -16.f;
#pragma unroll
  for (int q = 3; q >= 1; --q) {
    h[q] = h[q - 1];
    h[4 + q] = h[4 + q - 1];
    h[8 + q] = h[8 + q - 1];
  }
  h[0] = clampf((float)rho, -1.f, 2.f);
  h[4] = acc ? 1.f : 0.f;
  h[8] = clampf(ratio, -8.f, 1.f) / 8.f;
  float f[kMlpF];
  f[0] = (float)log10(s.lambda) / 4.f;
  f[1] = (float)log10((double)(s.iteration + 1)) / 2.f;
#pragma unroll
  for (int q = 0; q < kHist; ++q) f[2 + q] = h[q];
  f[14] = clampf(pratio, -16.f, 0.f) / 16.f;
  f[15] = 1.f;
  __syncwarp();
  if (lane < kHist) hk[lane] = h[lane];
  if (lane < kMlpF) feat[k * kMlpF + lane] = f[lane];
  int cls = -1;
  if (acc && w.theta) cls = mlp_policy_warp(w, f, lane);
  if (lane != 0) return;
  s.cost = cost;
  s.cost_new = cost_new;
  s.pred = pred;
  s.rho = rho;
  if (acc) {
    if (cls >= 0) {
      s.lambda *= mlp_multiplier(cls);
    } else {
      const double a = 2.0 * rho - 1.0;
      s.lambda *= fmax(1.0 / 3.0, 1.0 - a * a * a);
    }
    s.nu = 2.0;
    s.accepted = 1;
    if (ftol >= 0.0 && cost - cost_new <= ftol * cost) s.done = 1;
  } else {
    s.lambda *= s.nu;
    s.nu *= 2.0;
    s.accepted = 0;
  }
  if (s.lambda > 1e16) s.done = 1;
  if (s.lambda < 1e-30) s.lambda = 1e-30;
  s.iteration += 1;
  st[k] = s;
  if (s.done) atomicAdd(ndone, 1);
}

__global__ void lm_accept_kernel(LMTables t, const double* xnew, double* x, const qrkit_lm_state* st) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= t.N) return;
  if (st[t.col_prob[j]].accepted) x[j] = xnew[j];
}

inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

#define LM_LAUNCH(ctx, ...)                         \
  do {                                              \
    __VA_ARGS__;                                    \
    (ctx)->launches += 1;                           \
    QRKIT_CUDA_TRY(ctx, cudaGetLastError());        \
  } while (0)

// One LM iteration for every problem (all work on ctx->stream; no host synchronisation).
template <typename T>
qrkit_status lm_iteration(qrkit_ctx* ctx, double* x, int refine_steps, double ftol) {
  LM& L = *ctx->lm;
  const LMTables& t = L.t;
  cudaStream_t st = ctx->stream;
  qrkit_lm_state* S = (qrkit_lm_state*)L.state.ptr;
  T* J = (T*)L.J.ptr;
  T* Sv = (T*)L.S.ptr;
  T* b = (T*)L.b.ptr;
  T* p = (T*)L.p.ptr;
  double* d2 = (double*)L.d2.ptr;
  double* E = (double*)L.E.ptr;
  QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(d2 + t.NP, 0, (size_t)t.s * sizeof(double), st));
  QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(L.ndone.ptr, 0, sizeof(int), st));
  LM_LAUNCH(ctx, cf_eval_kernel<T><<<(unsigned)t.num_tiles, kTilePts, (size_t)L.sum_cols * sizeof(double), st>>>(
                     t, x, L.data, J, Sv, b, (int32_t*)L.start.ptr, d2, (double*)L.tile_cost.ptr, L.sum_cols));
  LM_LAUNCH(ctx, lm_damp_kernel<<<nblk(t.N, 256), 256, 0, st>>>(t, d2, S, E));
  qrkit_status rc = window_start_copy(ctx, (const int32_t*)L.start.ptr);
  if (rc != QRKIT_OK) return rc;
  if ((rc = composed_factor_scaled(ctx, J, Sv, E)) != QRKIT_OK) return rc;
  if ((rc = composed_solve(ctx, J, Sv, b, p, refine_steps)) != QRKIT_OK) return rc;
  double* xn = (double*)L.xnew.ptr;
  LM_LAUNCH(ctx, lm_xnew_kernel<T><<<nblk(t.N, 256), 256, 0, st>>>(t.N, x, p, xn));
  LM_LAUNCH(ctx, cf_trial_kernel<T><<<(unsigned)t.num_tiles, kTilePts, 0, st>>>(
                     t, xn, L.data, J, Sv, b, p, E, (const int32_t*)L.start.ptr, (double*)L.tile_new.ptr,
                     (double*)L.tile_pred.ptr));
  MlpDev w{};
  if (L.policy && ctx->mlp) {
    w.theta = (const float*)ctx->mlp->theta.ptr;
    w.wbf = (const __nv_bfloat16*)ctx->mlp->wbf.ptr;
  }
  LM_LAUNCH(ctx, lm_update_kernel<T><<<nblk(t.B * 32, 128), 128, 0, st>>>(
                     t, (const double*)L.tile_cost.ptr, (const double*)L.tile_new.ptr,
                     (const double*)L.tile_pred.ptr, E, p, S, ftol, (int*)L.ndone.ptr, w, (float*)L.hist.ptr,
                     (float*)L.feat.ptr));
  LM_LAUNCH(ctx, lm_accept_kernel<<<nblk(t.N, 256), 256, 0, st>>>(t, xn, x, S));
  return QRKIT_OK;
}

qrkit_status iterate(qrkit_ctx* ctx, double* x, int refine_steps, double ftol) {
  if (ctx->precision == QRKIT_FP64) return lm_iteration<double>(ctx, x, refine_steps, ftol);
  return lm_iteration<float>(ctx, x, refine_steps, ftol);
}

// Allocations and uploads of the composed factor happen here, outside any stream capture.
qrkit_status lm_prepare(qrkit_ctx* ctx) {
  LM& L = *ctx->lm;
  if (L.prepared) return QRKIT_OK;
  Composed& C = ctx->comp;
  C.damp = true;
  C.lam = 1.0;
  C.lam_half = 1.0;
  qrkit_status rc = composed_layout(ctx, elem_size(ctx));
  if (rc != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.D, (size_t)L.t.N * sizeof(double), "D")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.sq, (size_t)L.t.N * sizeof(double), "column sums")) != QRKIT_OK) return rc;
  L.prepared = true;
  return QRKIT_OK;
}

qrkit_status check_ready(qrkit_ctx* ctx, double* x, qrkit_lm_state* states, int refine_steps) {
  if (!ctx->lm) return fail(ctx, QRKIT_ESTATE, "no LM model planned (qrkit_lm_plan)");
  if (!x || !states) return fail(ctx, QRKIT_EINVAL, "x and states are required");
  if (refine_steps < 0 || refine_steps > 8) return fail(ctx, QRKIT_EINVAL, "refine_steps must be in [0, 8]");
  for (int64_t k = 0; k < ctx->lm->t.B; ++k)
    if (!(states[k].lambda > 0.0) || !(states[k].nu >= 1.0))
      return fail(ctx, QRKIT_EINVAL, "problem " + std::to_string(k) + ": lambda must be > 0 and nu >= 1");
  return QRKIT_OK;
}

qrkit_status read_status(qrkit_ctx* ctx) {
  QRKIT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  int h = 0;
  QRKIT_CUDA_TRY(ctx, cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    QRKIT_CUDA_TRY(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
    return fail(ctx, (qrkit_status)h, std::string("device reported ") + qrkit_status_string(h));
  }
  return QRKIT_OK;
}

}  // namespace
}  // namespace qrkit

using namespace qrkit;

extern "C" {

qrkit_status qrkit_lm_plan(qrkit_ctx* ctx, const qrkit_lm_problem* pr) {
  if (!ctx) return QRKIT_EINVAL;
  if (!pr) return fail(ctx, QRKIT_EINVAL, "null problem");
  if (pr->model != QRKIT_MODEL_CURVEFIT) return fail(ctx, QRKIT_EUNSUPPORTED, "unknown model");
  if (pr->num_problems < 1 || !pr->num_points || !pr->control_points || !pr->data)
    return fail(ctx, QRKIT_EINVAL, "num_problems >= 1, num_points, control_points and data are required");
  const int64_t B = pr->num_problems;
  std::vector<int64_t> p0(B + 1, 0), c0(B + 1, 0);
  for (int64_t k = 0; k < B; ++k) {
    if (pr->num_points[k] < 1) return fail(ctx, QRKIT_EINVAL, "problem " + std::to_string(k) + " has no points");
    if (pr->control_points[k] < 4)
      return fail(ctx, QRKIT_EINVAL, "problem " + std::to_string(k) + " needs at least 4 control points");
    p0[k + 1] = p0[k] + pr->num_points[k];
    c0[k + 1] = c0[k] + 2 * (int64_t)pr->control_points[k];
  }
  const int64_t NP = p0[B], s = c0[B];
  if (NP >= ((int64_t)1 << 31) || s >= ((int64_t)1 << 31))
    return fail(ctx, QRKIT_EUNSUPPORTED, "more than 2^31 points or shared columns");
  // block-angular structure: 2x1 blocks, windows of 8 shared columns, one segment per problem
  std::vector<uint8_t> n(NP, 2), m(NP, 1);
  std::vector<int32_t> ws(NP);
  std::vector<int64_t> seg_cols(B), seg_blocks(B);
  for (int64_t k = 0; k < B; ++k) {
    seg_cols[k] = c0[k + 1] - c0[k];
    seg_blocks[k] = p0[k + 1] - p0[k];
    for (int64_t i = p0[k]; i < p0[k + 1]; ++i) ws[i] = (int32_t)c0[k];
  }
  qrkit_structure st{};
  st.kind = QRKIT_STRUCT_BLOCKS;
  st.num_blocks = NP;
  st.block_rows = n.data();
  st.block_cols = m.data();
  st.coupled_kind = QRKIT_COUPLED_WINDOW;
  st.shared_cols = s;
  st.window = 8;
  st.window_start = ws.data();
  st.num_segments = B;
  st.segment_cols = seg_cols.data();
  st.segment_blocks = seg_blocks.data();
  qrkit_status rc = qrkit_plan(ctx, &st);   // releases any previous LM state
  if (rc != QRKIT_OK) return rc;
  ctx->lm = new LM();
  LM& L = *ctx->lm;
  L.t.B = B;
  L.t.NP = NP;
  L.t.s = s;
  L.t.N = NP + s;
  L.h_p0 = p0;
  L.h_c0 = c0;
  {
    int64_t widest = 0;
    for (size_t k = 0; k + 1 < c0.size(); ++k) widest = std::max<int64_t>(widest, c0[k + 1] - c0[k]);
    L.sum_cols = widest <= kEvalSumCols ? (int)widest : 0;
  }
  L.h_tile_p0.clear();
  L.h_prob_tile0.assign(B + 1, 0);
  std::vector<int32_t> tile_prob;
  for (int64_t k = 0; k < B; ++k) {
    L.h_prob_tile0[k] = (int64_t)L.h_tile_p0.size();
    for (int64_t q = p0[k]; q < p0[k + 1]; q += kTilePts) {
      L.h_tile_p0.push_back(q);
      tile_prob.push_back((int32_t)k);
    }
  }
  L.h_prob_tile0[B] = (int64_t)L.h_tile_p0.size();
  L.t.num_tiles = (int64_t)L.h_tile_p0.size();
  L.h_tile_p0.push_back(NP);
  std::vector<int32_t> col_prob(L.t.N);
  for (int64_t k = 0; k < B; ++k) {
    for (int64_t i = p0[k]; i < p0[k + 1]; ++i) col_prob[i] = (int32_t)k;
    for (int64_t c = c0[k]; c < c0[k + 1]; ++c) col_prob[NP + c] = (int32_t)k;
  }
  std::vector<int64_t> tabs;
  for (auto* v : {&p0, &c0, &L.h_tile_p0, &L.h_prob_tile0}) tabs.insert(tabs.end(), v->begin(), v->end());
  const size_t es = elem_size(ctx);
  auto up = [&](DevBuf& d, const void* h, size_t bytes, const char* what) -> qrkit_status {
    qrkit_status r = ensure(ctx, d, bytes, what);
    if (r != QRKIT_OK) return r;
    QRKIT_CUDA_TRY(ctx, cudaMemcpy(d.ptr, h, bytes, cudaMemcpyHostToDevice));
    return QRKIT_OK;
  };
  if ((rc = up(L.tabs, tabs.data(), tabs.size() * sizeof(int64_t), "LM tables")) != QRKIT_OK) return rc;
  if ((rc = up(L.tile_prob, tile_prob.data(), tile_prob.size() * sizeof(int32_t), "LM tiles")) != QRKIT_OK) return rc;
  if ((rc = up(L.col_prob, col_prob.data(), col_prob.size() * sizeof(int32_t), "LM columns")) != QRKIT_OK) return rc;
  const int64_t* tb = (const int64_t*)L.tabs.ptr;
  L.t.p0 = tb;
  L.t.c0 = tb + (B + 1);
  L.t.tile_p0 = tb + 2 * (B + 1);
  L.t.prob_tile0 = tb + 2 * (B + 1) + (L.t.num_tiles + 1);
  L.t.tile_prob = (const int32_t*)L.tile_prob.ptr;
  L.t.col_prob = (const int32_t*)L.col_prob.ptr;
  L.data = pr->data;
  const int64_t N = L.t.N, nt = L.t.num_tiles;
  if ((rc = ensure(ctx, L.J, (size_t)2 * NP * es, "LM J")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.S, (size_t)16 * NP * es, "LM S")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.b, (size_t)2 * NP * es, "LM b")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.p, (size_t)N * es, "LM p")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.start, (size_t)NP * sizeof(int32_t), "LM starts")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.d2, (size_t)N * sizeof(double), "LM norms")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.E, (size_t)N * sizeof(double), "LM damping")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.xnew, (size_t)N * sizeof(double), "LM trial point")) != QRKIT_OK) return rc;
  for (DevBuf* d : {&L.tile_cost, &L.tile_new, &L.tile_pred})
    if ((rc = ensure(ctx, *d, (size_t)nt * sizeof(double), "LM partial sums")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.state, (size_t)B * sizeof(qrkit_lm_state), "LM state")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.ndone, sizeof(int), "LM done count")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.hist, (size_t)B * kHist * sizeof(float), "LM history")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, L.feat, (size_t)B * kMlpF * sizeof(float), "LM features")) != QRKIT_OK) return rc;
  QRKIT_CUDA_TRY(ctx, cudaMemset(L.hist.ptr, 0, (size_t)B * kHist * sizeof(float)));
  QRKIT_CUDA_TRY(ctx, cudaMemset(L.feat.ptr, 0, (size_t)B * kMlpF * sizeof(float)));
  return QRKIT_OK;
}

qrkit_status qrkit_lm_linearize(qrkit_ctx* ctx, const double* x, void* J, void* S, void* b, int32_t* start) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->lm) return fail(ctx, QRKIT_ESTATE, "no LM model planned (qrkit_lm_plan)");
  if (!x) return fail(ctx, QRKIT_EINVAL, "x is required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  LM& L = *ctx->lm;
  const LMTables& t = L.t;
  cudaStream_t st = ctx->stream;
  double* d2 = (double*)L.d2.ptr;
  QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(d2 + t.NP, 0, (size_t)t.s * sizeof(double), st));
  if (ctx->precision == QRKIT_FP64)
    cf_eval_kernel<double><<<(unsigned)t.num_tiles, kTilePts, (size_t)L.sum_cols * sizeof(double), st>>>(
        t, x, L.data, (double*)L.J.ptr, (double*)L.S.ptr, (double*)L.b.ptr, (int32_t*)L.start.ptr, d2,
        (double*)L.tile_cost.ptr, L.sum_cols);
  else
    cf_eval_kernel<float><<<(unsigned)t.num_tiles, kTilePts, (size_t)L.sum_cols * sizeof(double), st>>>(
        t, x, L.data, (float*)L.J.ptr, (float*)L.S.ptr, (float*)L.b.ptr, (int32_t*)L.start.ptr, d2,
        (double*)L.tile_cost.ptr, L.sum_cols);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  const size_t es = elem_size(ctx);
  if (J) QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(J, L.J.ptr, (size_t)2 * t.NP * es, cudaMemcpyDeviceToDevice, st));
  if (S) QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(S, L.S.ptr, (size_t)16 * t.NP * es, cudaMemcpyDeviceToDevice, st));
  if (b) QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(b, L.b.ptr, (size_t)2 * t.NP * es, cudaMemcpyDeviceToDevice, st));
  if (start)
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(start, L.start.ptr, (size_t)t.NP * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return QRKIT_OK;
}

qrkit_status qrkit_lm_residual(qrkit_ctx* ctx, const double* x, double* f) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->lm) return fail(ctx, QRKIT_ESTATE, "no LM model planned (qrkit_lm_plan)");
  if (!x || !f) return fail(ctx, QRKIT_EINVAL, "x and f are required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  LM& L = *ctx->lm;
  cf_residual_kernel<<<(unsigned)L.t.num_tiles, kTilePts, 0, ctx->stream>>>(L.t, x, L.data, f);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

qrkit_status qrkit_lm_set_policy(qrkit_ctx* ctx, int use_mlp) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->lm) return fail(ctx, QRKIT_ESTATE, "no LM model planned (qrkit_lm_plan)");
  if (use_mlp && !ctx->mlp) return fail(ctx, QRKIT_ESTATE, "no MLP (qrkit_mlp_init)");
  LM& L = *ctx->lm;
  if (L.policy != (use_mlp != 0) && L.graph) {
    cudaGraphExecDestroy(L.graph);
    L.graph = nullptr;
  }
  L.policy = use_mlp != 0;
  return QRKIT_OK;
}

qrkit_status qrkit_lm_features(qrkit_ctx* ctx, float* features) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->lm) return fail(ctx, QRKIT_ESTATE, "no LM model planned (qrkit_lm_plan)");
  if (!features) return fail(ctx, QRKIT_EINVAL, "features is required");
  LM& L = *ctx->lm;
  QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(features, L.feat.ptr, (size_t)L.t.B * kMlpF * sizeof(float),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
  return QRKIT_OK;
}

qrkit_status qrkit_lm_step(qrkit_ctx* ctx, double* x, qrkit_lm_state* states, int refine_steps) {
  if (!ctx) return QRKIT_EINVAL;
  qrkit_status rc = check_ready(ctx, x, states, refine_steps);
  if (rc != QRKIT_OK) return rc;
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if ((rc = lm_prepare(ctx)) != QRKIT_OK) return rc;
  LM& L = *ctx->lm;
  const size_t sb = (size_t)L.t.B * sizeof(qrkit_lm_state);
  QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(L.state.ptr, states, sb, cudaMemcpyHostToDevice, ctx->stream));
  if ((rc = iterate(ctx, x, refine_steps, -1.0)) != QRKIT_OK) return rc;
  ctx->comp_factored = true;
  QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(states, L.state.ptr, sb, cudaMemcpyDeviceToHost, ctx->stream));
  return read_status(ctx);
}

qrkit_status qrkit_lm_run(qrkit_ctx* ctx, double* x, qrkit_lm_state* states, int max_iter, double ftol,
                          int refine_steps, int use_graph) {
  if (!ctx) return QRKIT_EINVAL;
  qrkit_status rc = check_ready(ctx, x, states, refine_steps);
  if (rc != QRKIT_OK) return rc;
  if (max_iter < 0) return fail(ctx, QRKIT_EINVAL, "max_iter must be >= 0");
  if (!(ftol >= 0.0)) return fail(ctx, QRKIT_EINVAL, "ftol must be >= 0");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if ((rc = lm_prepare(ctx)) != QRKIT_OK) return rc;
  LM& L = *ctx->lm;
  cudaStream_t st = ctx->stream;
  const size_t sb = (size_t)L.t.B * sizeof(qrkit_lm_state);
  QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(L.state.ptr, states, sb, cudaMemcpyHostToDevice, st));
  if (use_graph && (!L.graph || L.graph_refine != refine_steps || L.graph_ftol != ftol || L.graph_x != x)) {
    // capture one iteration (kernel arguments are fixed: x must stay the same buffer)
    if (L.graph) {
      cudaGraphExecDestroy(L.graph);
      L.graph = nullptr;
    }
    const int64_t before = ctx->launches;
    QRKIT_CUDA_TRY(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    rc = iterate(ctx, x, refine_steps, ftol);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc != QRKIT_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    const cudaError_t e2 = cudaGraphInstantiate(&L.graph, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaGraphInstantiate");
    L.graph_launches = ctx->launches - before;
    ctx->launches = before;
    L.graph_refine = refine_steps;
    L.graph_ftol = ftol;
    L.graph_x = x;
  }
  int done = 0;
  for (int it = 0; it < max_iter; ++it) {
    if (use_graph) {
      QRKIT_CUDA_TRY(ctx, cudaGraphLaunch(L.graph, st));
      ctx->launches += L.graph_launches;
    } else if ((rc = iterate(ctx, x, refine_steps, ftol)) != QRKIT_OK) {
      return rc;
    }
    if ((it + 1) % 8 == 0 || it + 1 == max_iter) {
      QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(&done, L.ndone.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
      QRKIT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
      if (done >= L.t.B) break;
    }
  }
  ctx->comp_factored = true;
  QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(states, L.state.ptr, sb, cudaMemcpyDeviceToHost, st));
  return read_status(ctx);
}

}  // extern "C"
