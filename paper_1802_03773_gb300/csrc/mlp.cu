// Damping-policy MLP: 16 features -> 64 -> 64 -> 8 logits over a grid of lambda multipliers
// (ReLU hidden layers, softmax cross-entropy, Adam).  Not in the paper: a learned alternative
// to the damping update of Sec. 2 / Sec. 5.2, with Nielsen's rule as its fallback.
//
// Parameters: one float32 vector [W1 (64x16) | b1 | W2 (64x64) | b2 | W3 (8x64) | b3] (the
// master copy Adam updates); the three weight matrices are also kept in bfloat16, which the
// forward and backward passes read (float32 accumulation, float32 activations and biases).
//
// Training step on n samples: tiles of 32 samples per CTA compute activations, the loss and
// all gradients in shared memory and write per-tile partial gradients; a second kernel sums
// the tiles in a fixed order (deterministic); Adam updates the master copy and refreshes the
// bfloat16 weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "internal.h"
#include "mlp_policy.cuh"

namespace qrkit {

namespace {

constexpr int F = kMlpF, H = kMlpH, C = kMlpC;
constexpr int oW1 = 0, ob1 = oW1 + H * F, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + C * H;
constexpr int P = ob3 + C;
constexpr int NW = H * F + H * H + C * H;   // bfloat16 weights
constexpr int kTile = 32;                   // samples per CTA
constexpr int kThreads = 256;
static_assert(P == kMlpParams, "parameter layout");

__global__ void mlp_round_kernel(const float* theta, __nv_bfloat16* wbf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NW) return;
  int src;
  if (e < H * F) src = oW1 + e;
  else if (e < H * F + H * H) src = oW2 + (e - H * F);
  else src = oW3 + (e - H * F - H * H);
  wbf[e] = __float2bfloat16_rn(theta[src]);
}

// Forward (and with BWD the backward pass) for one tile of samples.
template <bool BWD>
__global__ void __launch_bounds__(kThreads)
mlp_tile_kernel(const float* theta, const __nv_bfloat16* wbf, const float* X, const int32_t* labels, int64_t n,
                float* logits, float* partial, float* loss_part) {
  __shared__ float sW1[H * F], sW2[H * H], sW3[C * H], sb[H + H + C];
  __shared__ float sX[kTile * F], sA1[kTile * H], sA2[kTile * H], sZ[kTile * C];
  const int tid = threadIdx.x;
  const int64_t s0 = (int64_t)blockIdx.x * kTile;
  for (int e = tid; e < H * F; e += kThreads) sW1[e] = __bfloat162float(wbf[e]);
  for (int e = tid; e < H * H; e += kThreads) sW2[e] = __bfloat162float(wbf[H * F + e]);
  for (int e = tid; e < C * H; e += kThreads) sW3[e] = __bfloat162float(wbf[H * F + H * H + e]);
  for (int e = tid; e < H; e += kThreads) {
    sb[e] = theta[ob1 + e];
    sb[H + e] = theta[ob2 + e];
  }
  if (tid < C) sb[2 * H + tid] = theta[ob3 + tid];
  for (int e = tid; e < kTile * F; e += kThreads) {
    const int64_t s = s0 + e / F;
    sX[e] = s < n ? X[s * F + (e % F)] : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < kTile * H; e += kThreads) {
    const int s = e / H, h = e % H;
    float a = sb[h];
#pragma unroll
    for (int f = 0; f < F; ++f) a = fmaf(sW1[h * F + f], sX[s * F + f], a);
    sA1[e] = a;
  }
  __syncthreads();
  for (int e = tid; e < kTile * H; e += kThreads) {
    const int s = e / H, h = e % H;
    float a = sb[H + h];
    for (int k = 0; k < H; ++k) a = fmaf(sW2[h * H + k], fmaxf(sA1[s * H + k], 0.f), a);
    sA2[e] = a;
  }
  __syncthreads();
  if (tid < kTile * C) {
    const int s = tid / C, c = tid % C;
    float z = sb[2 * H + c];
    for (int k = 0; k < H; ++k) z = fmaf(sW3[c * H + k], fmaxf(sA2[s * H + k], 0.f), z);
    sZ[tid] = z;
    if (!BWD && s0 + s < n) logits[(s0 + s) * C + c] = z;
  }
  __syncthreads();
  if (!BWD) return;
  // softmax cross-entropy: sZ becomes dL/dz (mean over the n samples)
  __shared__ float sLoss[kTile];
  if (tid < kTile) {
    const int s = tid;
    float l = 0.f;
    if (s0 + s < n) {
      float zmax = sZ[s * C];
      for (int c = 1; c < C; ++c) zmax = fmaxf(zmax, sZ[s * C + c]);
      float den = 0.f;
      for (int c = 0; c < C; ++c) den += expf(sZ[s * C + c] - zmax);
      const int lab = labels[s0 + s];
      l = -(sZ[s * C + lab] - zmax - logf(den));
      for (int c = 0; c < C; ++c) {
        const float pr = expf(sZ[s * C + c] - zmax) / den;
        sZ[s * C + c] = (pr - (c == lab ? 1.f : 0.f)) / (float)n;
      }
    } else {
      for (int c = 0; c < C; ++c) sZ[s * C + c] = 0.f;
    }
    sLoss[s] = l;
  }
  __syncthreads();
  float* g = partial + (int64_t)blockIdx.x * P;
  if (tid == 0) {
    float l = 0.f;
    for (int s = 0; s < kTile; ++s) l += sLoss[s];
    loss_part[blockIdx.x] = l / (float)n;
  }
  // dW3, db3
  for (int e = tid; e < C * H + C; e += kThreads) {
    if (e < C * H) {
      const int c = e / H, k = e % H;
      float a = 0.f;
      for (int s = 0; s < kTile; ++s) a = fmaf(sZ[s * C + c], fmaxf(sA2[s * H + k], 0.f), a);
      g[oW3 + e] = a;
    } else {
      const int c = e - C * H;
      float a = 0.f;
      for (int s = 0; s < kTile; ++s) a += sZ[s * C + c];
      g[ob3 + c] = a;
    }
  }
  __syncthreads();
  // dA2 = (W3^T dz) * relu'(A2), in place of A2
  for (int e = tid; e < kTile * H; e += kThreads) {
    const int s = e / H, h = e % H;
    float a = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) a = fmaf(sW3[c * H + h], sZ[s * C + c], a);
    sA2[e] = sA2[e] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // dW2, db2
  for (int e = tid; e < H * H + H; e += kThreads) {
    if (e < H * H) {
      const int h = e / H, k = e % H;
      float a = 0.f;
      for (int s = 0; s < kTile; ++s) a = fmaf(sA2[s * H + h], fmaxf(sA1[s * H + k], 0.f), a);
      g[oW2 + e] = a;
    } else {
      const int h = e - H * H;
      float a = 0.f;
      for (int s = 0; s < kTile; ++s) a += sA2[s * H + h];
      g[ob2 + h] = a;
    }
  }
  __syncthreads();
  // dA1 = (W2^T dA2) * relu'(A1), in place of A1
  for (int e = tid; e < kTile * H; e += kThreads) {
    const int s = e / H, k = e % H;
    float a = 0.f;
    for (int h = 0; h < H; ++h) a = fmaf(sW2[h * H + k], sA2[s * H + h], a);
    sA1[e] = sA1[e] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // dW1, db1
  for (int e = tid; e < H * F + H; e += kThreads) {
    if (e < H * F) {
      const int k = e / F, f = e % F;
      float a = 0.f;
      for (int s = 0; s < kTile; ++s) a = fmaf(sA1[s * H + k], sX[s * F + f], a);
      g[oW1 + e] = a;
    } else {
      const int k = e - H * F;
      float a = 0.f;
      for (int s = 0; s < kTile; ++s) a += sA1[s * H + k];
      g[ob1 + k] = a;
    }
  }
}

__global__ void mlp_reduce_kernel(const float* partial, const float* loss_part, int tiles, float* grad,
                                  float* loss) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < P) {
    float a = 0.f;
    for (int t = 0; t < tiles; ++t) a += partial[(int64_t)t * P + j];
    grad[j] = a;
  }
  if (j == P) {
    float a = 0.f;
    for (int t = 0; t < tiles; ++t) a += loss_part[t];
    *loss = a;
  }
}

__global__ void mlp_adam_kernel(float* theta, const float* grad, float* m, float* v, float lr, float c1, float c2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const float gj = grad[j];
  const float mj = 0.9f * m[j] + 0.1f * gj;
  const float vj = 0.999f * v[j] + 0.001f * gj * gj;
  m[j] = mj;
  v[j] = vj;
  theta[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + 1e-8f);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void release_mlp(Mlp*& m) {
  if (!m) return;
  for (DevBuf* b : {&m->theta, &m->wbf, &m->m, &m->v, &m->grad, &m->partial, &m->loss_part, &m->loss}) release(*b);
  delete m;
  m = nullptr;
}

static qrkit_status mlp_refresh(qrkit_ctx* ctx) {
  Mlp& M = *ctx->mlp;
  mlp_round_kernel<<<nblk(NW, 256), 256, 0, ctx->stream>>>((const float*)M.theta.ptr, (__nv_bfloat16*)M.wbf.ptr);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

}  // namespace qrkit

using namespace qrkit;

extern "C" {

qrkit_status qrkit_mlp_init(qrkit_ctx* ctx, const float* params) {
  if (!ctx) return QRKIT_EINVAL;
  if (!params) return fail(ctx, QRKIT_EINVAL, "params are required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (!ctx->mlp) ctx->mlp = new Mlp();
  Mlp& M = *ctx->mlp;
  qrkit_status rc;
  if ((rc = ensure(ctx, M.theta, P * sizeof(float), "MLP parameters")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, M.wbf, NW * sizeof(__nv_bfloat16), "MLP bf16 weights")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, M.m, P * sizeof(float), "Adam m")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, M.v, P * sizeof(float), "Adam v")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, M.grad, P * sizeof(float), "MLP gradient")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, M.loss, sizeof(float), "MLP loss")) != QRKIT_OK) return rc;
  QRKIT_CUDA_TRY(ctx, cudaMemcpy(M.theta.ptr, params, P * sizeof(float), cudaMemcpyHostToDevice));
  QRKIT_CUDA_TRY(ctx, cudaMemset(M.m.ptr, 0, P * sizeof(float)));
  QRKIT_CUDA_TRY(ctx, cudaMemset(M.v.ptr, 0, P * sizeof(float)));
  M.step = 0;
  return mlp_refresh(ctx);
}

qrkit_status qrkit_mlp_params(qrkit_ctx* ctx, float* params) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->mlp) return fail(ctx, QRKIT_ESTATE, "no MLP (qrkit_mlp_init)");
  if (!params) return fail(ctx, QRKIT_EINVAL, "params is required");
  QRKIT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  QRKIT_CUDA_TRY(ctx, cudaMemcpy(params, ctx->mlp->theta.ptr, P * sizeof(float), cudaMemcpyDeviceToHost));
  return QRKIT_OK;
}

qrkit_status qrkit_mlp_forward(qrkit_ctx* ctx, const float* X, int64_t n, float* logits) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->mlp) return fail(ctx, QRKIT_ESTATE, "no MLP (qrkit_mlp_init)");
  if (n < 0 || (n > 0 && (!X || !logits))) return fail(ctx, QRKIT_EINVAL, "X and logits are required");
  if (n == 0) return QRKIT_OK;
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  Mlp& M = *ctx->mlp;
  mlp_tile_kernel<false><<<nblk(n, kTile), kThreads, 0, ctx->stream>>>(
      (const float*)M.theta.ptr, (const __nv_bfloat16*)M.wbf.ptr, X, nullptr, n, logits, nullptr, nullptr);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

qrkit_status qrkit_mlp_train_step(qrkit_ctx* ctx, const float* X, const int32_t* labels, int64_t n, float lr,
                                  float* loss_out, float* grad_out) {
  if (!ctx) return QRKIT_EINVAL;
  if (!ctx->mlp) return fail(ctx, QRKIT_ESTATE, "no MLP (qrkit_mlp_init)");
  if (n < 1 || !X || !labels) return fail(ctx, QRKIT_EINVAL, "X, labels and n >= 1 are required");
  if (!(lr >= 0.f)) return fail(ctx, QRKIT_EINVAL, "lr must be >= 0");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  Mlp& M = *ctx->mlp;
  cudaStream_t st = ctx->stream;
  const int64_t tiles = (n + kTile - 1) / kTile;
  if (tiles > (1 << 20)) return fail(ctx, QRKIT_EUNSUPPORTED, "batch too large");
  qrkit_status rc;
  if ((rc = ensure(ctx, M.partial, (size_t)tiles * P * sizeof(float), "MLP partial gradients")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, M.loss_part, (size_t)tiles * sizeof(float), "MLP partial loss")) != QRKIT_OK) return rc;
  mlp_tile_kernel<true><<<(unsigned)tiles, kThreads, 0, st>>>((const float*)M.theta.ptr,
                                                               (const __nv_bfloat16*)M.wbf.ptr, X, labels, n,
                                                               nullptr, (float*)M.partial.ptr,
                                                               (float*)M.loss_part.ptr);
  mlp_reduce_kernel<<<nblk(P + 1, 256), 256, 0, st>>>((const float*)M.partial.ptr, (const float*)M.loss_part.ptr,
                                                       (int)tiles, (float*)M.grad.ptr, (float*)M.loss.ptr);
  ctx->launches += 2;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  if (grad_out)
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(grad_out, M.grad.ptr, P * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (lr > 0.f) {
    M.step += 1;
    const float c1 = 1.f - powf(0.9f, (float)M.step), c2 = 1.f - powf(0.999f, (float)M.step);
    mlp_adam_kernel<<<nblk(P, 256), 256, 0, st>>>((float*)M.theta.ptr, (const float*)M.grad.ptr, (float*)M.m.ptr,
                                                   (float*)M.v.ptr, lr, c1, c2);
    ctx->launches += 1;
    QRKIT_CUDA_TRY(ctx, cudaGetLastError());
    if ((rc = mlp_refresh(ctx)) != QRKIT_OK) return rc;
  }
  if (loss_out) {
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(loss_out, M.loss.ptr, sizeof(float), cudaMemcpyDeviceToHost, st));
    QRKIT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  }
  return QRKIT_OK;
}

}  // extern "C"
