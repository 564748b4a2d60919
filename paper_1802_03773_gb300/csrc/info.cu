// Diagnostics of a block-diagonal solve (the result record a caller reads after a solve): the
// residual norm ||b - J p||, the norm of the optimality residual J^T (b - J p) - lambda D^2 p
// (zero at the exact minimiser of Eq. 2, where (J^T J + lambda D^2) p = J^T b, Eq. 1) with its
// natural scale, and the refinement's selection count and most steps taken.
//
// One thread per block accumulates its block's squared norms in double; each CTA adds its
// threads' values in a fixed order and writes one partial per quantity; a second kernel adds the
// partials in order, so the result does not depend on scheduling.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "block_tasks.cuh"
#include "internal.h"

namespace qrkit {
namespace {

constexpr int kInfoThreads = 256;
constexpr int kInfoQty = 5;   // ||r||^2, ||g||^2, ||J||_F^2, ||p||^2, ||b||^2

template <typename T>
__global__ void __launch_bounds__(kInfoThreads) info_blocks_kernel(const T* J, const T* b, const T* p, const T* D,
                                                                 double lambda, const uint8_t* nn, const uint8_t* mm,
                                                                 const int64_t* vo, const int64_t* ro,
                                                                 const int64_t* co, int64_t K, double* part) {
  __shared__ double red[kInfoQty][kInfoThreads];
  const int64_t i = (int64_t)blockIdx.x * kInfoThreads + threadIdx.x;
  double q[kInfoQty] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (i < K) {
    const int n = nn[i], m = mm[i];
    const T* A = J + vo[i];
    const T* bi = b + ro[i];
    const T* x = p + co[i];
    double r[16];
    for (int k = 0; k < n; ++k) {
      double s = (double)bi[k];
      for (int j = 0; j < m; ++j) s -= (double)A[(int64_t)j * n + k] * (double)x[j];
      r[k] = s;
      q[0] += s * s;
      q[4] += (double)bi[k] * (double)bi[k];
    }
    for (int j = 0; j < m; ++j) {
      double g = 0.0, c2 = 0.0;
      for (int k = 0; k < n; ++k) {
        const double a = (double)A[(int64_t)j * n + k];
        g += a * r[k];
        c2 += a * a;
      }
      double d = D ? (double)D[co[i] + j] : sqrt(c2);
      if (!D && d == 0.0) d = 1.0;
      g -= lambda * d * d * (double)x[j];
      q[1] += g * g;
      q[2] += c2;
      q[3] += (double)x[j] * (double)x[j];
    }
  }
  for (int t = 0; t < kInfoQty; ++t) red[t][threadIdx.x] = q[t];
  __syncthreads();
  for (int h = kInfoThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int t = 0; t < kInfoQty; ++t) red[t][threadIdx.x] += red[t][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < kInfoQty) part[(int64_t)blockIdx.x * kInfoQty + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void info_sum_kernel(const double* part, int64_t parts, double* out) {
  if (threadIdx.x >= kInfoQty) return;
  double s = 0.0;
  for (int64_t k = 0; k < parts; ++k) s += part[k * kInfoQty + threadIdx.x];
  out[threadIdx.x] = s;
}

// Terms of the predicted decrease 1/2 p^T (lambda D^2 p + J^T b) = 1/2 (lambda ||D p||^2 +
// b^T J p) of a composed plan: thread i < K takes block i's rows (b^T J p over them, the coupled
// columns included) and its columns' lambda D_j^2 p_j^2; thread K + c takes shared column c.
template <typename T>
__global__ void __launch_bounds__(kInfoThreads) pred_kernel(ComposedView<T> V, const T* b, const T* p,
                                                          const double* D, double lambda, double* part) {
  __shared__ double red[2][kInfoThreads];
  const int64_t i = (int64_t)blockIdx.x * kInfoThreads + threadIdx.x;
  double bjp = 0.0, dp = 0.0;
  if (i < V.K) {
    const int n = V.n[i], m = V.m[i];
    const int64_t c0 = V.col_off[i], r0 = V.row_off[i];
    const T* Ji = V.J + V.val_off[i];
    const int64_t st = V.coupled == QRKIT_COUPLED_WINDOW ? V.start[i] : 0;
    for (int r = 0; r < n; ++r) {
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc += (double)Ji[j * n + r] * (double)p[c0 + j];
      if (V.coupled == QRKIT_COUPLED_DENSE) {
        for (int c = 0; c < V.s; ++c) acc += (double)V.S[(int64_t)c * V.rows + r0 + r] * (double)p[V.nb + c];
      } else if (V.coupled == QRKIT_COUPLED_WINDOW) {
        for (int t = 0; t < V.w; ++t)
          if (st + t < V.s) acc += (double)V.S[r0 * V.w + (int64_t)t * n + r] * (double)p[V.nb + st + t];
      }
      bjp += (double)b[r0 + r] * acc;
    }
    for (int j = 0; j < m; ++j) {
      const double v = D[c0 + j] * (double)p[c0 + j];
      dp += v * v;
    }
  } else if (i < V.K + V.s) {
    const int64_t c = V.nb + (i - V.K);
    const double v = D[c] * (double)p[c];
    dp += v * v;
  }
  red[0][threadIdx.x] = bjp;
  red[1][threadIdx.x] = lambda * dp;
  __syncthreads();
  for (int h = kInfoThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) part[(int64_t)blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void pred_sum_kernel(const double* part, int64_t parts, double* out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, c = 0.0;
  for (int64_t k = 0; k < parts; ++k) {
    a += part[2 * k];
    c += part[2 * k + 1];
  }
  out[0] = 0.5 * (c + a);
}

template <typename T>
qrkit_status pred_typed(qrkit_ctx* ctx, const void* J, const void* S, const void* b, const void* p, double* pred) {
  ComposedView<T> V = composed_view<T>(ctx, J, S);
  const int64_t parts = (V.K + V.s + kInfoThreads - 1) / kInfoThreads;
  DevBuf buf;
  qrkit_status st = ensure(ctx, buf, (size_t)(2 * parts + 1) * sizeof(double), "predicted decrease");
  if (st != QRKIT_OK) return st;
  double* part = (double*)buf.ptr;
  pred_kernel<T><<<(unsigned)parts, kInfoThreads, 0, ctx->stream>>>(V, (const T*)b, (const T*)p,
                                                                   (const double*)ctx->comp.D.ptr, ctx->comp.lam, part);
  pred_sum_kernel<<<1, 32, 0, ctx->stream>>>(part, parts, part + 2 * parts);
  ctx->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(pred, part + 2 * parts, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  release(buf);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "predicted decrease");
  return QRKIT_OK;
}

}  // namespace
}  // namespace qrkit

extern "C" qrkit_status qrkit_lm_trial(qrkit_ctx* ctx, const void* J, const void* S, const void* b, const void* D,
                                       double lambda, int refine_steps, void* p, double* pred) {
  using namespace qrkit;
  if (!ctx) return QRKIT_EINVAL;
  if (!pred || !b || !p) return fail(ctx, QRKIT_EINVAL, "b, p and pred are required");
  qrkit_status st = qrkit_factor(ctx, J, S, D, lambda);
  if (st != QRKIT_OK) return st;
  if ((st = qrkit_solve(ctx, b, p, refine_steps)) != QRKIT_OK) return st;
  if (ctx->precision == QRKIT_FP64) return pred_typed<double>(ctx, J, S, b, p, pred);
  return pred_typed<float>(ctx, J, S, b, p, pred);
}

extern "C" qrkit_status qrkit_nielsen_update(double rho, double* lambda, double* nu, int32_t* accepted) {
  if (!lambda || !nu) return QRKIT_EINVAL;
  if (!(*lambda > 0.0) || !(*nu > 0.0)) return QRKIT_EINVAL;
  if (rho > 0.0) {
    const double t = 2.0 * rho - 1.0;
    const double f = 1.0 - t * t * t;
    *lambda *= f > 1.0 / 3.0 ? f : 1.0 / 3.0;
    *nu = 2.0;
    if (accepted) *accepted = 1;
  } else {
    *lambda *= *nu;
    *nu *= 2.0;
    if (accepted) *accepted = 0;
  }
  return QRKIT_OK;
}

extern "C" qrkit_status qrkit_get_info(qrkit_ctx* ctx, const void* J, const void* b, const void* p, const void* D,
                                       double lambda, qrkit_info* out) {
  using namespace qrkit;
  if (!ctx) return QRKIT_EINVAL;
  if (!out || !J || !b || !p) return fail(ctx, QRKIT_EINVAL, "J, b, p and out are required");
  if (!(lambda >= 0.0)) return fail(ctx, QRKIT_EINVAL, "lambda must be >= 0");
  const Plan& P = ctx->plan;
  if (!P.valid || P.s.kind != QRKIT_STRUCT_BLOCKS || P.s.coupled_kind != QRKIT_COUPLED_NONE)
    return fail(ctx, QRKIT_EUNSUPPORTED, "qrkit_get_info needs a block-diagonal plan");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int64_t parts = (P.K + kInfoThreads - 1) / kInfoThreads;
  DevBuf buf;
  qrkit_status st = ensure(ctx, buf, (size_t)(parts + 1) * kInfoQty * sizeof(double), "info partials");
  if (st != QRKIT_OK) return st;
  double* part = (double*)buf.ptr;
  double* sums = part + parts * kInfoQty;
  if (ctx->precision == QRKIT_FP64)
    info_blocks_kernel<double><<<(unsigned)parts, kInfoThreads, 0, ctx->stream>>>(
        (const double*)J, (const double*)b, (const double*)p, (const double*)D, lambda, (const uint8_t*)P.d_n.ptr,
        (const uint8_t*)P.d_m.ptr, (const int64_t*)P.d_val_off.ptr, (const int64_t*)P.d_row_off.ptr,
        (const int64_t*)P.d_col_off.ptr, P.K, part);
  else
    info_blocks_kernel<float><<<(unsigned)parts, kInfoThreads, 0, ctx->stream>>>(
        (const float*)J, (const float*)b, (const float*)p, (const float*)D, lambda, (const uint8_t*)P.d_n.ptr,
        (const uint8_t*)P.d_m.ptr, (const int64_t*)P.d_val_off.ptr, (const int64_t*)P.d_row_off.ptr,
        (const int64_t*)P.d_col_off.ptr, P.K, part);
  info_sum_kernel<<<1, 32, 0, ctx->stream>>>(part, parts, sums);
  ctx->launches += 2;
  cudaError_t e = cudaGetLastError();
  double h[kInfoQty] = {0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  int cnt[kTaskKeys + 1] = {0};
  const bool stats = ctx->refine_stats && ctx->ws.tcount.ptr && P.mapping == 0;
  if (e == cudaSuccess && stats)
    e = cudaMemcpyAsync(cnt, ctx->ws.tcount.ptr, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  release(buf);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "qrkit_get_info");
  out->residual_norm = sqrt(h[0]);
  out->optimality_norm = sqrt(h[1]);
  const double jF = sqrt(h[2]);
  out->optimality_scale = jF * (jF * sqrt(h[3]) + sqrt(h[4]));
  if (stats) {
    int64_t sel = 0;
    for (int k = 0; k < kTaskKeys; ++k)
      sel += std::min<int64_t>(cnt[k], P.key_off[k + 1] - P.key_off[k]);
    out->refined_blocks = sel;
    out->refine_steps_max = cnt[kTaskKeys];
  } else {
    out->refined_blocks = -1;
    out->refine_steps_max = -1;
  }
  return QRKIT_OK;
}
