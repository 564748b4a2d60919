// Dense least squares min ||A x - b|| by Householder QR (Sec. 2) in one CTA: the merge step of a
// shared block whose rows are split over several GPUs (each GPU's reduced block summarised by
// its s x s triangle; the stacked triangles, plus the shared columns' damping rows, are factored
// once).  Column k: the norm of A[k:, k] by a block reduction, the reflector (v[0] = 1,
// beta = -sign(x0) ||x||), then one warp per trailing column (and the right-hand side) applies
// it with the lanes over rows; back-substitution by one warp.  A is copied to a workspace of the
// context first (the caller's A is not changed).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace qrkit {
namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// A: M x N column-major (ld M) in the workspace, c: M; x: N out; res2: squared residual norm.
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) dense_lstsq_kernel(T* A, int64_t M, int N, T* c, T* x,
                                                                 double* res2, int* status) {
  __shared__ double red[kThreads / 32];
  __shared__ T coef[3];   // tau, beta, 1 / (alpha - beta)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < N; ++k) {
    T* col = A + (int64_t)k * M;
    double sq = 0.0;
    for (int64_t i = k + 1 + tid; i < M; i += kThreads) sq += (double)col[i] * (double)col[i];
    sq = warp_sum(sq);
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) t += red[w];
      const T alpha = col[k];
      const T nrm = (T)sqrt((double)alpha * (double)alpha + t);
      T tau = T(0), beta = alpha, scale = T(0);
      if (nrm != T(0)) {
        beta = alpha >= T(0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = T(1) / (alpha - beta);
      }
      coef[0] = tau;
      coef[1] = beta;
      coef[2] = scale;
    }
    __syncthreads();
    const T tau = coef[0], scale = coef[2];
    for (int64_t i = k + 1 + tid; i < M; i += kThreads) col[i] *= scale;
    __syncthreads();
    // trailing columns j = k + 1 .. N - 1 and the rhs (j = N), one warp each
    for (int j = k + 1 + warp; j <= N; j += kThreads / 32) {
      T* cj = j < N ? A + (int64_t)j * M : c;
      T w = T(0);
      for (int64_t i = k + 1 + lane; i < M; i += 32) w += col[i] * cj[i];
      w = warp_sum(w) + cj[k];
      w *= tau;
      if (lane == 0) cj[k] -= w;
      for (int64_t i = k + 1 + lane; i < M; i += 32) cj[i] -= col[i] * w;
    }
    __syncthreads();
    if (tid == 0) col[k] = coef[1];
    __syncthreads();
  }
  if (warp == 0) {
    double r2 = 0.0;
    for (int64_t i = N + lane; i < M; i += 32) r2 += (double)c[i] * (double)c[i];
    r2 = warp_sum(r2);
    if (lane == 0 && res2) *res2 = r2;
    for (int k = N - 1; k >= 0; --k) {
      T part = T(0);
      for (int j = k + 1 + lane; j < N; j += 32) part += A[(int64_t)j * M + k] * x[j];
      part = warp_sum(part);
      if (lane == 0) {
        const T rkk = A[(int64_t)k * M + k];
        if (rkk == T(0) && status) atomicCAS(status, 0, (int)QRKIT_ESINGULAR);
        x[k] = (c[k] - part) / rkk;
      }
      __syncwarp();
    }
  }
}

template <typename T>
qrkit_status dense_typed(qrkit_ctx* ctx, int64_t M, int64_t N, const void* A, int64_t lda, const void* b,
                         void* x, double* res2) {
  DevBuf& W = ctx->comp.dense_ws;
  const size_t es = sizeof(T);
  qrkit_status st = ensure(ctx, W, (size_t)(M * N + M) * es + sizeof(double), "dense least squares");
  if (st != QRKIT_OK) return st;
  T* Aw = (T*)W.ptr;
  T* cw = Aw + M * N;
  double* r2 = reinterpret_cast<double*>(cw + M);
  QRKIT_CUDA_TRY(ctx, cudaMemcpy2DAsync(Aw, (size_t)M * es, A, (size_t)lda * es, (size_t)M * es, (size_t)N,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
  QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(cw, b, (size_t)M * es, cudaMemcpyDeviceToDevice, ctx->stream));
  dense_lstsq_kernel<T><<<1, kThreads, 0, ctx->stream>>>(Aw, M, (int)N, cw, (T*)x, r2, ctx->d_status);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  if (res2) {
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(res2, r2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    QRKIT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return QRKIT_OK;
}

}  // namespace
}  // namespace qrkit

extern "C" qrkit_status qrkit_dense_lstsq(qrkit_ctx* ctx, int64_t M, int64_t N, const void* A, int64_t lda,
                                          const void* b, void* x, double* res2) {
  using namespace qrkit;
  if (!ctx) return QRKIT_EINVAL;
  if (!A || !b || !x) return fail(ctx, QRKIT_EINVAL, "A, b and x are required");
  if (N < 1 || M < N || lda < M) return fail(ctx, QRKIT_EINVAL, "need 1 <= N <= M <= lda");
  if (N > 1024 || M * N > (int64_t)1 << 24)
    return fail(ctx, QRKIT_EUNSUPPORTED, "the one-CTA dense solve takes N <= 1024 and M N <= 2^24");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (ctx->precision == QRKIT_FP64) return dense_typed<double>(ctx, M, N, A, lda, b, x, res2);
  return dense_typed<float>(ctx, M, N, A, lda, b, x, res2);
}
