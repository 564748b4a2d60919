// Damping-policy MLP: layout constants and the one-warp inference used inside the LM update
// kernel (header so that every translation unit inlines it; no relocatable device code).
#pragma once

#include <cuda_bf16.h>
#include <math.h>

namespace qrkit {

constexpr int kMlpF = 16;   // features
constexpr int kMlpH = 64;   // hidden width
constexpr int kMlpC = 8;    // classes: lambda multipliers
constexpr int kMlpParams = kMlpH * kMlpF + kMlpH + kMlpH * kMlpH + kMlpH + kMlpC * kMlpH + kMlpC;

// lambda multiplier of each class (the step after an accepted trial uses lambda * multiplier)
__device__ __forceinline__ double mlp_multiplier(int c) {
  switch (c) {
    case 0: return 1e-2;
    case 1: return 1e-1;
    case 2: return 1.0 / 3.0;
    case 3: return 0.5;
    case 4: return 1.0;
    case 5: return 2.0;
    case 6: return 4.0;
    default: return 10.0;
  }
}

struct MlpDev {
  const float* theta = nullptr;          // float32 parameters (biases read from here)
  const __nv_bfloat16* wbf = nullptr;    // W1 | W2 | W3 in bfloat16
};

// Inference for one problem by one warp (the features in every lane): argmax class.
__device__ __forceinline__ int mlp_policy_warp(const MlpDev& w, const float* feat, int lane) {
  constexpr int F = kMlpF, H = kMlpH, C = kMlpC;
  constexpr int ob1 = H * F, ob2 = ob1 + H + H * H, ob3 = ob2 + H + C * H;
  float h1[2], h2[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int h = lane + 32 * q;
    float a = w.theta[ob1 + h];
#pragma unroll
    for (int f = 0; f < F; ++f) a = fmaf(__bfloat162float(w.wbf[h * F + f]), feat[f], a);
    h1[q] = fmaxf(a, 0.f);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int h = lane + 32 * q;
    float a = w.theta[ob2 + h];
    for (int k = 0; k < H; ++k) {
      const float v0 = __shfl_sync(0xffffffffu, h1[0], k & 31);
      const float v1 = __shfl_sync(0xffffffffu, h1[1], k & 31);
      a = fmaf(__bfloat162float(w.wbf[H * F + h * H + k]), k < 32 ? v0 : v1, a);
    }
    h2[q] = fmaxf(a, 0.f);
  }
  const int c = lane < C ? lane : 0;
  float a = w.theta[ob3 + c];
  for (int k = 0; k < H; ++k) {
    const float v0 = __shfl_sync(0xffffffffu, h2[0], k & 31);
    const float v1 = __shfl_sync(0xffffffffu, h2[1], k & 31);
    a = fmaf(__bfloat162float(w.wbf[H * F + H * H + c * H + k]), k < 32 ? v0 : v1, a);
  }
  float bz = lane < C ? a : -INFINITY;
  int best = lane < C ? lane : C;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const float oz = __shfl_xor_sync(0xffffffffu, bz, d);
    const int ob = __shfl_xor_sync(0xffffffffu, best, d);
    if (oz > bz || (oz == bz && ob < best)) {
      bz = oz;
      best = ob;
    }
  }
  return best;
}

}  // namespace qrkit
