// Composed QR of the damped block-angular system (Sec. 4.1, 4.2, 4.5, 5.1, 5.2):
//   P_r [J; lambda^(1/2) D] = [[blkdiag(B_i), C], [0, lambda^(1/2) D_S]],
//   B_i = [J_i; lambda^(1/2) D_i], C_i = [S_i; 0]  (row interleave, Sec. 4.5 / 5.2).
// Steps: D = column norms (Sec. 5.2); per block Q_i R_i = qr(B_i) (Sec. 4.1) with Q_i^T
// applied to C_i (Sec. 4.2): top rows -> R12_i, bottom rows -> reduced shared block; the
// reduced block [stacked bottoms; lambda^(1/2) D_S] is factored by TSQR (tall-skinny QR:
// row tiles factored in parallel, their R's stacked and factored again); solve R p = Q^T b
// by back-substitution (Sec. 5.1); optional refinement with FP64 residuals.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "device_util.cuh"
#include "internal.h"

namespace qrkit {
namespace {

constexpr int kMaxRows = 16;   // augmented rows per block
constexpr int kMaxCols = 8;    // columns per block
constexpr int kChunk = 8;      // coupled columns processed per pass
constexpr int kTileThreads = 256;

__device__ __forceinline__ void record(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---- column norms D = diag(J^T J)^(1/2) (Sec. 5.2), accumulated in double ----
template <typename T>
__global__ void colnorm_blocks_kernel(ComposedView<T> V, double* sq) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V.K) return;
  const int n = V.n[i], m = V.m[i];
  const T* J = V.J + V.val_off[i];
  for (int j = 0; j < m; ++j) {
    double s = 0;
    for (int r = 0; r < n; ++r) {
      const double x = (double)J[j * n + r];
      s += x * x;
    }
    sq[V.col_off[i] + j] = s;
  }
}

// Dense S (column-major, ld = rows of J): squared column norms in two deterministic passes.
// Pass 1, one CTA per (chunk of kNormRows rows, shared column): strided per-thread sums, then
// the warps' sums in warp order; pass 2, one thread per column adds its chunks in order.
constexpr int kNormRows = 8192;
constexpr int kNormThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kNormThreads) colnorm_dense_part_kernel(ComposedView<T> V, double* part,
                                                                          int64_t nchunk) {
  __shared__ double ws[kNormThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * kNormRows;
  const int64_t r1 = r0 + kNormRows < V.rows ? r0 + kNormRows : V.rows;
  for (int64_t col = blockIdx.y; col < V.s; col += gridDim.y) {
    const T* c = V.S + col * V.rows;
    double s = 0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kNormThreads) {
      const double x = (double)c[r];
      s += x * x;
    }
    for (int d = 16; d >= 1; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) ws[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < kNormThreads / 32; ++w) t += ws[w];
      part[col * nchunk + blockIdx.x] = t;
    }
    __syncthreads();   // ws is reused by the next column
  }
}

__global__ void colnorm_dense_sum_kernel(const double* part, int64_t nchunk, int64_t s, double* sq) {
  const int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (col >= s) return;
  double t = 0;
  for (int64_t k = 0; k < nchunk; ++k) t += part[col * nchunk + k];
  sq[col] = t;
}

template <typename T>
__global__ void colnorm_window_kernel(ComposedView<T> V, double* sq) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V.K) return;
  const int n = V.n[i];
  const T* C = V.S + V.row_off[i] * V.w;   // block i: n x w column-major
  for (int t = 0; t < V.w; ++t) {
    double s = 0;
    for (int r = 0; r < n; ++r) {
      const double x = (double)C[t * n + r];
      s += x * x;
    }
    const int64_t col = V.start[i] + t;
    if (s != 0.0 && col < V.s) atomicAdd(&sq[V.nb + col], s);
  }
}

__global__ void finalize_norms_kernel(const double* sq, double* D, int64_t N) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double d = sqrt(sq[j]);
  D[j] = d == 0.0 ? 1.0 : d;   // zero column norm -> 1 (MINPACK convention)
}

// ---- per-block factor (Sec. 4.1) with Q_i^T applied to the coupled columns (Sec. 4.2) ----
// One thread per block; the augmented block B_i = [J_i; lambda^(1/2) D_i] (na x m) is held
// column-major in local arrays.  Outputs: factor Fa (na x m, V below / R on and above the
// diagonal), tau, R12 rows (m x w) and the reduced rows (na - m rows).
// Small blocks (at most NA augmented rows and MM columns, e.g. the 2 x 1 blocks of curve and
// ellipse fits): the same factorization as the general path below, with every loop unrolled to
// the compile-time bounds (runtime sizes as guards), so the block, its reflectors and a chunk
// of coupled columns stay in registers instead of local memory.
template <typename T, int NA, int MM>
__device__ __forceinline__ void block_factor_small(const ComposedView<T>& V, const FactorOut<T>& O, int64_t i, int n,
                                                   int m) {
  const int na = n + (O.damp ? m : 0);
  const T* J = V.J + V.val_off[i];
  T B[MM][NA];
#pragma unroll
  for (int j = 0; j < MM; ++j)
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      T v = T(0);
      if (j < m) {
        if (r < n) v = J[j * n + r];
        else if (O.damp && r - n == j) v = (T)(O.lam_half * O.D[V.col_off[i] + j]);
      }
      B[j][r] = v;
    }
  T tau[MM];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < MM; ++k) {
    tau[k] = T(0);
    if (k < m) {
      T sq = 0;
#pragma unroll
      for (int r = 0; r < NA; ++r)
        if (r > k && r < na) sq += B[k][r] * B[k][r];
      const T alpha = B[k][k];
      const T norm = sqrt(alpha * alpha + sq);
      T beta = 0, t = 0, scale = 0;
      if (norm != T(0)) {
        beta = alpha >= T(0) ? -norm : norm;
        t = (beta - alpha) / beta;
        scale = T(1) / (alpha - beta);
      } else {
        bad = true;
      }
#pragma unroll
      for (int r = 0; r < NA; ++r)
        if (r > k) B[k][r] *= scale;
      B[k][k] = beta;
      tau[k] = t;
#pragma unroll
      for (int j = k + 1; j < MM; ++j) {
        if (j < m) {
          T w = B[j][k];
#pragma unroll
          for (int r = 0; r < NA; ++r)
            if (r > k && r < na) w += B[k][r] * B[j][r];
          w *= t;
          B[j][k] -= w;
#pragma unroll
          for (int r = 0; r < NA; ++r)
            if (r > k && r < na) B[j][r] -= w * B[k][r];
        }
      }
    }
  }
  if (bad) record(O.status, QRKIT_ESINGULAR);
  T* F = O.Fa + O.aug_off[i];
#pragma unroll
  for (int j = 0; j < MM; ++j)
#pragma unroll
    for (int r = 0; r < NA; ++r)
      if (j < m && r < na) F[j * na + r] = B[j][r];
#pragma unroll
  for (int k = 0; k < MM; ++k)
    if (k < m) O.tau[V.col_off[i] + k] = tau[k];
  if (V.coupled == QRKIT_COUPLED_NONE) return;
  const int64_t red0 = O.red_off[i];
  if constexpr (sizeof(T) == 4 && NA == 3 && MM == 1) {
    // the 2 x 1 point blocks of curve fits with windows of 8 (damped): the window, R12 and
    // the two reduced rows are moved by 16-byte loads and stores (all 32-byte aligned)
    if (V.coupled == QRKIT_COUPLED_WINDOW && V.w == 8 && n == 2 && m == 1 && na == 3 &&
        (reinterpret_cast<uintptr_t>(V.S) & 15) == 0) {   // the caller's S 16-byte aligned
      const float4* src = reinterpret_cast<const float4*>(V.S + V.row_off[i] * 8);   // 2 x 8 column-major
      float sv[16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 v = src[q];
        sv[4 * q] = v.x;
        sv[4 * q + 1] = v.y;
        sv[4 * q + 2] = v.z;
        sv[4 * q + 3] = v.w;
      }
      float r12[8], x1[8], x2[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        // column c of the augmented window: rows (S[0][c], S[1][c], 0); reflector k = 0
        const float y0 = sv[2 * c], y1 = sv[2 * c + 1];
        float w = y0 + B[0][1] * y1;   // row 2 of the column is 0
        w *= tau[0];
        r12[c] = y0 - w;
        x1[c] = y1 - w * B[0][1];
        x2[c] = -w * B[0][2];
      }
      float4* dr = reinterpret_cast<float4*>(O.R12 + V.col_off[i] * 8);
      dr[0] = make_float4(r12[0], r12[1], r12[2], r12[3]);
      dr[1] = make_float4(r12[4], r12[5], r12[6], r12[7]);
      float4* dx = reinterpret_cast<float4*>(O.Xw + red0 * 8);
      dx[0] = make_float4(x1[0], x1[1], x1[2], x1[3]);
      dx[1] = make_float4(x1[4], x1[5], x1[6], x1[7]);
      dx[2] = make_float4(x2[0], x2[1], x2[2], x2[3]);
      dx[3] = make_float4(x2[4], x2[5], x2[6], x2[7]);
      O.Xstart[red0] = V.start[i];
      O.Xstart[red0 + 1] = V.start[i];
      return;
    }
  }
  for (int c0 = 0; c0 < V.w; c0 += kChunk) {
    const int cw = min(kChunk, V.w - c0);
    T C[kChunk][NA];
#pragma unroll
    for (int c = 0; c < kChunk; ++c)
#pragma unroll
      for (int r = 0; r < NA; ++r) {
        T v = T(0);
        if (c < cw && r < n) {
          if (V.coupled == QRKIT_COUPLED_DENSE) v = V.S[(int64_t)(c0 + c) * V.rows + V.row_off[i] + r];
          else v = V.S[V.row_off[i] * V.w + (int64_t)(c0 + c) * n + r];
        }
        C[c][r] = v;
      }
#pragma unroll
    for (int k = 0; k < MM; ++k) {
      if (k < m) {
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
          T w = C[c][k];
#pragma unroll
          for (int r = 0; r < NA; ++r)
            if (r > k && r < na) w += B[k][r] * C[c][r];
          w *= tau[k];
          C[c][k] -= w;
#pragma unroll
          for (int r = 0; r < NA; ++r)
            if (r > k && r < na) C[c][r] -= w * B[k][r];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kChunk; ++c) {
      if (c < cw) {
#pragma unroll
        for (int r = 0; r < NA; ++r) {
          if (r < m) {
            O.R12[(V.col_off[i] + r) * (int64_t)V.w + c0 + c] = C[c][r];
          } else if (r < na) {
            const int64_t row = red0 + (r - m);
            if (V.coupled == QRKIT_COUPLED_DENSE) {
              O.X0[(int64_t)(c0 + c) * O.ld0 + row] = C[c][r];
            } else {
              O.Xw[row * V.w + c0 + c] = C[c][r];
              if (c0 + c == 0) O.Xstart[row] = V.start[i];
            }
          }
        }
      }
    }
  }
}

// Plans whose blocks all fit (NA, MM) run this kernel (its register needs are those of the
// small blocks only).
template <typename T, int NA, int MM>
__global__ void block_factor_small_kernel(ComposedView<T> V, FactorOut<T> O) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V.K) return;
  block_factor_small<T, NA, MM>(V, O, i, V.n[i], V.m[i]);
}

template <typename T>
__global__ void block_factor_kernel(ComposedView<T> V, FactorOut<T> O) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V.K) return;
  const int n = V.n[i], m = V.m[i];
  const int na = n + (O.damp ? m : 0);
  T B[kMaxRows * kMaxCols];
  const T* J = V.J + V.val_off[i];
  for (int j = 0; j < m; ++j) {
    for (int r = 0; r < n; ++r) B[j * na + r] = J[j * n + r];
    if (O.damp)
      for (int r = 0; r < m; ++r)
        B[j * na + n + r] = (r == j) ? (T)(O.lam_half * O.D[V.col_off[i] + j]) : T(0);
  }
  T tau[kMaxCols];
  bool bad = false;
  for (int k = 0; k < m; ++k) {
    T* x = B + k * na;
    T sq = 0;
    for (int r = k + 1; r < na; ++r) sq += x[r] * x[r];
    const T alpha = x[k];
    const T norm = sqrt(alpha * alpha + sq);
    T beta = 0, t = 0, scale = 0;
    if (norm != T(0)) {
      beta = alpha >= T(0) ? -norm : norm;
      t = (beta - alpha) / beta;
      scale = T(1) / (alpha - beta);
    } else {
      bad = true;
    }
    for (int r = k + 1; r < na; ++r) x[r] *= scale;
    x[k] = beta;
    tau[k] = t;
    for (int j = k + 1; j < m; ++j) {
      T* y = B + j * na;
      T w = y[k];
      for (int r = k + 1; r < na; ++r) w += x[r] * y[r];
      w *= t;
      y[k] -= w;
      for (int r = k + 1; r < na; ++r) y[r] -= w * x[r];
    }
  }
  if (bad) record(O.status, QRKIT_ESINGULAR);
  T* F = O.Fa + O.aug_off[i];
  for (int e = 0; e < na * m; ++e) F[e] = B[e];
  for (int k = 0; k < m; ++k) O.tau[V.col_off[i] + k] = tau[k];
  // coupled columns, kChunk at a time
  if (V.coupled == QRKIT_COUPLED_NONE) return;
  const int64_t red0 = O.red_off[i];
  for (int c0 = 0; c0 < V.w; c0 += kChunk) {
    const int cw = min(kChunk, V.w - c0);
    T C[kMaxRows * kChunk];
    for (int c = 0; c < cw; ++c) {
      for (int r = 0; r < n; ++r) {
        T v;
        if (V.coupled == QRKIT_COUPLED_DENSE) v = V.S[(int64_t)(c0 + c) * V.rows + V.row_off[i] + r];
        else v = V.S[V.row_off[i] * V.w + (int64_t)(c0 + c) * n + r];
        C[c * na + r] = v;
      }
      for (int r = n; r < na; ++r) C[c * na + r] = 0;
    }
    for (int k = 0; k < m; ++k) {
      const T* x = B + k * na;
      for (int c = 0; c < cw; ++c) {
        T* y = C + c * na;
        T w = y[k];
        for (int r = k + 1; r < na; ++r) w += x[r] * y[r];
        w *= tau[k];
        y[k] -= w;
        for (int r = k + 1; r < na; ++r) y[r] -= w * x[r];
      }
    }
    for (int c = 0; c < cw; ++c) {
      for (int r = 0; r < m; ++r) O.R12[(V.col_off[i] + r) * (int64_t)V.w + c0 + c] = C[c * na + r];
      for (int r = m; r < na; ++r) {
        const int64_t row = red0 + (r - m);
        if (V.coupled == QRKIT_COUPLED_DENSE) {
          O.X0[(int64_t)(c0 + c) * O.ld0 + row] = C[c * na + r];
        } else {
          O.Xw[row * V.w + c0 + c] = C[c * na + r];
          if (c0 + c == 0) O.Xstart[row] = V.start[i];
        }
      }
    }
  }
}

// Damping rows of the shared columns, appended below the stacked bottoms (dense case).
template <typename T>
__global__ void reduced_damping_kernel(T* X0, int64_t ld0, int64_t row0, int s, const double* D,
                                       int64_t nb, double lam_half) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)s * s) return;
  const int j = (int)(e / s), c = (int)(e % s);
  X0[(int64_t)c * ld0 + row0 + j] = (c == j) ? (T)(lam_half * D[nb + j]) : T(0);
}

// ---- TSQR tile factor: one CTA per row tile of a level matrix (column-major, ld) ----
// Householder QR of the tile in shared memory; V below / R on and above the diagonal are
// written back in place, tau to taus[tile * s + k], and the tile's R rows (upper
// triangle, zeros below) to the next level's rows [tile * s, tile * s + min(r, s)).
template <typename T>
__global__ void __launch_bounds__(kTileThreads)
tsqr_tile_kernel(T* X, int64_t ld, int64_t M, int s, int tile_rows, T* taus, T* Xn, int64_t ldn,
                 int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);                 // tile_rows x s, ld = tile_rows
  T* red = A + (size_t)tile_rows * s;                    // 32 partials
  T* sh = red + 32;                                      // [0] tau, [1] beta, [2] scale
  const int64_t r0 = (int64_t)blockIdx.x * tile_rows;
  const int r = (int)(M - r0 < (int64_t)tile_rows ? M - r0 : (int64_t)tile_rows);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  for (int e = tid; e < r * s; e += blockDim.x) {
    const int c = e / r, i = e % r;
    A[c * tile_rows + i] = X[(int64_t)c * ld + r0 + i];
  }
  __syncthreads();
  const int kmax = min(r, s);
  for (int k = 0; k < kmax; ++k) {
    T* x = A + k * tile_rows;
    if (warp == 0) {
      T sq = 0;
      for (int i = k + 1 + lane; i < r; i += 32) sq += x[i] * x[i];
      for (int d = 16; d >= 1; d >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, d);
      if (lane == 0) {
        const T alpha = x[k];
        const T norm = sqrt(alpha * alpha + sq);
        T beta = 0, t = 0, scale = 0;
        if (norm != T(0)) {
          beta = alpha >= T(0) ? -norm : norm;
          t = (beta - alpha) / beta;
          scale = T(1) / (alpha - beta);
        }
        // a zero column inside a tile is not a singular R: a tile of stacked R rows can
        // start below the diagonal; the final R_S is checked by the back-substitution
        sh[0] = t;
        sh[1] = beta;
        sh[2] = scale;
      }
      __syncwarp();
      const T scale = sh[2];
      for (int i = k + 1 + lane; i < r; i += 32) x[i] *= scale;
    }
    __syncthreads();
    const T t = sh[0];
    for (int j = k + 1 + warp; j < s; j += nwarps) {
      T* y = A + j * tile_rows;
      T w = 0;
      for (int i = k + 1 + lane; i < r; i += 32) w += x[i] * y[i];
      for (int d = 16; d >= 1; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
      w = (w + y[k]) * t;
      if (lane == 0) y[k] -= w;
      for (int i = k + 1 + lane; i < r; i += 32) y[i] -= w * x[i];
    }
    if (tid == 0) {
      x[k] = sh[1];
      taus[(int64_t)blockIdx.x * s + k] = t;
    }
    __syncthreads();
  }
  for (int e = tid; e < r * s; e += blockDim.x) {
    const int c = e / r, i = e % r;
    X[(int64_t)c * ld + r0 + i] = A[c * tile_rows + i];
  }
  if (Xn) {
    const int64_t n0 = (int64_t)blockIdx.x * s;
    for (int e = tid; e < kmax * s; e += blockDim.x) {
      const int c = e / kmax, i = e % kmax;
      Xn[(int64_t)c * ldn + n0 + i] = (c >= i) ? A[c * tile_rows + i] : T(0);
    }
  }
}

// Q_tile^T applied to a level's rhs segment; the top min(r, s) entries go to the next level, and
// with column panels the others to the next panel's first level (row down0 + tile (tile_rows - s)).
template <typename T>
__global__ void __launch_bounds__(kTileThreads)
tsqr_apply_qt_kernel(const T* X, int64_t ld, int64_t M, int s, int tile_rows, const T* taus,
                     T* rhs, T* rhs_next, T* rhs_down, int64_t down0) {
  __shared__ T red[32];
  const int64_t r0 = (int64_t)blockIdx.x * tile_rows;
  const int r = (int)(M - r0 < (int64_t)tile_rows ? M - r0 : (int64_t)tile_rows);
  const int kmax = min(r, s);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* y = rhs + r0;
  for (int k = 0; k < kmax; ++k) {
    const T* x = X + (int64_t)k * ld + r0;
    T w = 0;
    for (int i = k + 1 + tid; i < r; i += blockDim.x) w += x[i] * y[i];
    for (int d = 16; d >= 1; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
    if (lane == 0) red[warp] = w;
    __syncthreads();
    if (warp == 0) {
      T v = lane < (int)(blockDim.x >> 5) ? red[lane] : T(0);
      for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
      if (lane == 0) red[0] = v;
    }
    __syncthreads();
    const T wt = (red[0] + y[k]) * taus[(int64_t)blockIdx.x * s + k];
    __syncthreads();
    if (tid == 0) y[k] -= wt;
    for (int i = k + 1 + tid; i < r; i += blockDim.x) y[i] -= wt * x[i];
    __syncthreads();
  }
  if (rhs_next)
    for (int i = tid; i < kmax; i += blockDim.x) rhs_next[(int64_t)blockIdx.x * s + i] = y[i];
  if (rhs_down)   // column panels: the rows below the tile's R rows, for the next panel
    for (int i = kmax + tid; i < r; i += blockDim.x)
      rhs_down[down0 + (int64_t)blockIdx.x * (tile_rows - s) + (i - kmax)] = y[i];
}

// Per-block Q_i^T [b_i; 0]: top m -> ctop, bottom -> reduced rhs rows.  NA > 0: every block has
// at most NA augmented rows and MM columns (loops unrolled to those bounds, registers only).
template <typename T, int NA = 0, int MM = 0>
__global__ void block_apply_qt_kernel(ComposedView<T> V, FactorOut<T> O, const T* b, T* rhs0) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V.K) return;
  if constexpr (NA > 0) {
    const int n = V.n[i], m = V.m[i];
    const int na = n + (O.damp ? m : 0);
    T y[NA];
#pragma unroll
    for (int r = 0; r < NA; ++r) y[r] = r < n ? b[V.row_off[i] + r] : T(0);
    const T* F = O.Fa + O.aug_off[i];
#pragma unroll
    for (int k = 0; k < MM; ++k) {
      if (k < m) {
        T w = y[k];
#pragma unroll
        for (int r = 0; r < NA; ++r)
          if (r > k && r < na) w += F[k * na + r] * y[r];
        w *= O.tau[V.col_off[i] + k];
        y[k] -= w;
#pragma unroll
        for (int r = 0; r < NA; ++r)
          if (r > k && r < na) y[r] -= w * F[k * na + r];
      }
    }
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      if (r < m) O.ctop[V.col_off[i] + r] = y[r];
      else if (rhs0 && r < na) rhs0[O.red_off[i] + (r - m)] = y[r];
    }
    return;
  }
  const int n = V.n[i], m = V.m[i];
  const int na = n + (O.damp ? m : 0);
  T y[kMaxRows];
  for (int r = 0; r < n; ++r) y[r] = b[V.row_off[i] + r];
  for (int r = n; r < na; ++r) y[r] = 0;
  const T* F = O.Fa + O.aug_off[i];
  for (int k = 0; k < m; ++k) {
    const T* x = F + k * na;
    T w = y[k];
    for (int r = k + 1; r < na; ++r) w += x[r] * y[r];
    w *= O.tau[V.col_off[i] + k];
    y[k] -= w;
    for (int r = k + 1; r < na; ++r) y[r] -= w * x[r];
  }
  for (int r = 0; r < m; ++r) O.ctop[V.col_off[i] + r] = y[r];
  if (rhs0)
    for (int r = m; r < na; ++r) rhs0[O.red_off[i] + (r - m)] = y[r];
}

// The s x s triangle R_S is solved by one CTA with a thread per row (s <= kTriMax).
constexpr int kTriMax = 1024;
static inline unsigned tri_threads(int s) { return (unsigned)(s <= 32 ? 32 : (s + 31) / 32 * 32); }

template <typename T>
__device__ __forceinline__ T block_warp_sum(T v) {
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// R_S x = c (upper triangular, column-major with ld), optionally x += result (x may be c).
// Columns are eliminated from the last: once x_k is known, every row above subtracts R_ik x_k,
// so each column is read once, coalesced, and the next one is loaded a step ahead.
template <typename T>
__global__ void __launch_bounds__(kTriMax) dense_backsub_kernel(const T* R, int64_t ld, int s, const T* c, T* x,
                                                                int accumulate, int* status) {
  __shared__ T xs[2];
  const int i = threadIdx.x;
  T yi = i < s ? c[i] : T(0);
  T rcur = i < s ? R[(int64_t)(s - 1) * ld + i] : T(0);   // column s - 1
  for (int k = s - 1; k >= 0; --k) {
    const T rnext = i < k ? R[(int64_t)(k - 1) * ld + i] : T(0);
    if (i == k) {
      if (rcur == T(0)) record(status, QRKIT_ESINGULAR);
      xs[k & 1] = yi / rcur;
    }
    __syncthreads();
    const T xk = xs[k & 1];
    if (i < k) yi -= rcur * xk;
    else if (i == k) yi = xk;
    rcur = rnext;
  }
  if (i < s) x[i] = accumulate ? x[i] + yi : yi;
}

// R_S^T h = g (forward substitution), g given in double: h_k = (g_k - sum_{i<k} R_ik h_i) / R_kk,
// the sum over column k of R (coalesced, loaded a step ahead) reduced over the CTA.
template <typename T>
__global__ void __launch_bounds__(kTriMax) dense_fwdsub_rt_kernel(const T* R, int64_t ld, int s, const double* g,
                                                                  T* h) {
  __shared__ T part_s[2][32];
  __shared__ T hs[2];
  const int i = threadIdx.x, lane = i & 31, warp = i >> 5, nw = (int)(blockDim.x >> 5);
  T hi = T(0);
  T rcur = i < 1 && s > 0 ? R[0] : T(0);                          // column 0
  T dnext = s > 0 && i == 0 ? R[0] : T(0), gnext = s > 0 && i == 0 ? (T)g[0] : T(0);
  for (int k = 0; k < s; ++k) {
    const T rnext = (k + 1 < s && i <= k + 1) ? R[(int64_t)(k + 1) * ld + i] : T(0);
    const T dk = dnext, gk = gnext;   // thread 0: R_kk and g_k
    if (i == 0 && k + 1 < s) {
      dnext = R[(int64_t)(k + 1) * ld + k + 1];
      gnext = (T)g[k + 1];
    }
    const T p = block_warp_sum<T>(i < k ? rcur * hi : T(0));
    if (lane == 0) part_s[k & 1][warp] = p;
    __syncthreads();
    if (warp == 0) {
      const T q = block_warp_sum<T>(lane < nw ? part_s[k & 1][lane] : T(0));
      if (lane == 0) hs[k & 1] = (gk - q) / dk;
    }
    __syncthreads();
    if (i == k) hi = hs[k & 1];
    rcur = rnext;
  }
  if (i < s) h[i] = hi;
}

// Per-block R_i x_i = rhs_i - R12_i x_S; rhs from ctop (T) or from a double vector.  NA > 0:
// every block has at most NA augmented rows and MM columns (registers only).
template <typename T, int NA = 0, int MM = 0>
__global__ void block_backsub_kernel(ComposedView<T> V, FactorOut<T> O, const T* rhs_t,
                                     const T* xS, T* x, int accumulate) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= V.K) return;
  if constexpr (NA > 0) {
    const int n = V.n[i], m = V.m[i];
    const int na = n + (O.damp ? m : 0);
    const int64_t c0 = V.col_off[i];
    const int64_t st = V.coupled == QRKIT_COUPLED_WINDOW ? V.start[i] : 0;
    T y[MM];
#pragma unroll
    for (int k = 0; k < MM; ++k) {
      T v = T(0);
      if (k < m) {
        v = rhs_t[c0 + k];
        if (V.coupled != QRKIT_COUPLED_NONE && xS) {
          const T* r12 = O.R12 + (c0 + k) * (int64_t)V.w;
          for (int t = 0; t < V.w; ++t)
            if (st + t < V.s) v -= r12[t] * xS[st + t];
        }
      }
      y[k] = v;
    }
    const T* F = O.Fa + O.aug_off[i];
#pragma unroll
    for (int k = MM - 1; k >= 0; --k) {
      if (k < m) {
        T v = y[k];
#pragma unroll
        for (int j = k + 1; j < MM; ++j)
          if (j < m) v -= F[j * na + k] * y[j];
        y[k] = v / F[k * na + k];
      }
    }
#pragma unroll
    for (int k = 0; k < MM; ++k)
      if (k < m) x[c0 + k] = accumulate ? x[c0 + k] + y[k] : y[k];
    return;
  }
  const int n = V.n[i], m = V.m[i];
  const int na = n + (O.damp ? m : 0);
  const int64_t c0 = V.col_off[i];
  T y[kMaxCols];
  for (int k = 0; k < m; ++k) {
    T v = rhs_t[c0 + k];
    if (V.coupled != QRKIT_COUPLED_NONE && xS) {
      const int64_t st = V.coupled == QRKIT_COUPLED_WINDOW ? V.start[i] : 0;
      const T* r12 = O.R12 + (c0 + k) * (int64_t)V.w;
      for (int t = 0; t < V.w; ++t)
        if (st + t < V.s) v -= r12[t] * xS[st + t];
    }
    y[k] = v;
  }
  const T* F = O.Fa + O.aug_off[i];
  for (int k = m - 1; k >= 0; --k) {
    T v = y[k];
    for (int j = k + 1; j < m; ++j) v -= F[j * na + k] * y[j];
    y[k] = v / F[k * na + k];
  }
  for (int k = 0; k < m; ++k) x[c0 + k] = accumulate ? x[c0 + k] + y[k] : y[k];
}

// ---- refinement: g = J^T (b - J p) - lambda D^2 p in double ----
constexpr int kCtaSumCols = 4096;   // dense S: shared columns summed per CTA in shared memory
constexpr int kWinSumCols = 2048;   // windowed S: the column range of a CTA summed in shared memory

template <typename T>
__device__ __forceinline__ void resid_g_block(ComposedView<T> V, const T* b, const T* p, const double* D,
                                              double lam, double* g, double* gS, int64_t goff, int64_t i) {
  const int n = V.n[i], m = V.m[i];
  const int64_t c0 = V.col_off[i], r0 = V.row_off[i];
  const T* J = V.J + V.val_off[i];
  const int64_t st = V.coupled == QRKIT_COUPLED_WINDOW ? V.start[i] : 0;
  double res[kMaxRows];
  for (int r = 0; r < n; ++r) {
    double acc = (double)b[r0 + r];
    for (int j = 0; j < m; ++j) acc -= (double)J[j * n + r] * (double)p[c0 + j];
    if (V.coupled == QRKIT_COUPLED_DENSE) {
      for (int c = 0; c < V.s; ++c)
        acc -= (double)V.S[(int64_t)c * V.rows + r0 + r] * (double)p[V.nb + c];
    } else if (V.coupled == QRKIT_COUPLED_WINDOW) {
      for (int t = 0; t < V.w; ++t)
        if (st + t < V.s) acc -= (double)V.S[r0 * V.w + (int64_t)t * n + r] * (double)p[V.nb + st + t];
    }
    res[r] = acc;
  }
  for (int j = 0; j < m; ++j) {
    double acc = 0;
    for (int r = 0; r < n; ++r) acc += (double)J[j * n + r] * res[r];
    const double d = D[c0 + j];
    g[c0 + j] = acc - lam * d * d * (double)p[c0 + j];
  }
  if (V.coupled == QRKIT_COUPLED_DENSE) {
    for (int c = 0; c < V.s; ++c) {
      double acc = 0;
      for (int r = 0; r < n; ++r) acc += (double)V.S[(int64_t)c * V.rows + r0 + r] * res[r];
      if (acc != 0.0) atomicAdd(&gS[c], acc);
    }
  } else if (V.coupled == QRKIT_COUPLED_WINDOW) {
    for (int t = 0; t < V.w; ++t) {
      double acc = 0;
      for (int r = 0; r < n; ++r) acc += (double)V.S[r0 * V.w + (int64_t)t * n + r] * res[r];
      if (acc != 0.0 && st + t < V.s) atomicAdd(&gS[st + t - goff], acc);
    }
  }
}

// Compensated float accumulation (Dot2, Ogita-Rump-Oishi): (sh + sl) += a x with the product's
// rounding error from an FMA and the sum's from TwoSum (Knuth).
__device__ __forceinline__ void dot2_acc(float& sh, float& sl, float a, float x) {
  const float p = __fmul_rn(a, x);
  const float pe = __fmaf_rn(a, x, -p);
  float t, e;
  dev::two_sum(sh, p, t, e);
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(e, pe));
}

// resid_g_small for float data: the residual b - J p - S p_S and the sums J^T r, S^T r in
// compensated float arithmetic (as if in twice the working precision) instead of FP64, whose
// rate on this part is a small fraction of FP32's; each sum is rounded to double once, for g
// and the column accumulation.
template <int NR, int MM>
__device__ __forceinline__ void resid_g_small_f32(const ComposedView<float>& V, const float* b, const float* p,
                                                  const double* D, double lam, double* g, double* gS, int64_t goff,
                                                  int64_t i) {
  const int n = V.n[i], m = V.m[i];
  const int64_t c0 = V.col_off[i], r0 = V.row_off[i];
  const float* J = V.J + V.val_off[i];
  const int64_t st = V.coupled == QRKIT_COUPLED_WINDOW ? V.start[i] : 0;
  if constexpr (MM == 1 && NR >= 2) {
    // the 2 x 1 point blocks of curve fits with windows of 8: the window (2 x 8 column-major,
    // 32-byte aligned in a 16-byte aligned S) by four 16-byte loads
    if (V.coupled == QRKIT_COUPLED_WINDOW && V.w == 8 && n == 2 && m == 1 &&
        (reinterpret_cast<uintptr_t>(V.S) & 15) == 0) {
      const float4* s4 = reinterpret_cast<const float4*>(V.S + r0 * 8);
      float sv[16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 v = s4[q];
        sv[4 * q] = v.x;
        sv[4 * q + 1] = v.y;
        sv[4 * q + 2] = v.z;
        sv[4 * q + 3] = v.w;
      }
      const float p0 = p[c0];
      float ps[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) ps[t] = st + t < V.s ? p[V.nb + st + t] : 0.f;
      float rh2[2], rl2[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float sh = b[r0 + r], sl = 0.f;
        dot2_acc(sh, sl, -J[r], p0);
#pragma unroll
        for (int t = 0; t < 8; ++t) dot2_acc(sh, sl, -sv[2 * t + r], ps[t]);
        rh2[r] = sh;
        rl2[r] = sl;
      }
      {
        float ah = 0.f, al = 0.f;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          dot2_acc(ah, al, J[r], rh2[r]);
          al = __fmaf_rn(J[r], rl2[r], al);
        }
        const double d = D[c0];
        g[c0] = ((double)ah + (double)al) - lam * d * d * (double)p0;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float ah = 0.f, al = 0.f;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          dot2_acc(ah, al, sv[2 * t + r], rh2[r]);
          al = __fmaf_rn(sv[2 * t + r], rl2[r], al);
        }
        const double acc = (double)ah + (double)al;
        if (acc != 0.0 && st + t < V.s) atomicAdd(&gS[st + t - goff], acc);
      }
      return;
    }
  }
  float pj[MM], rh[NR], rl[NR];
#pragma unroll
  for (int j = 0; j < MM; ++j) pj[j] = j < m ? p[c0 + j] : 0.f;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    float sh = 0.f, sl = 0.f;
    if (r < n) {
      sh = b[r0 + r];
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (j < m) dot2_acc(sh, sl, -J[j * n + r], pj[j]);
      if (V.coupled == QRKIT_COUPLED_DENSE) {
        for (int c = 0; c < V.s; ++c) dot2_acc(sh, sl, -V.S[(int64_t)c * V.rows + r0 + r], p[V.nb + c]);
      } else if (V.coupled == QRKIT_COUPLED_WINDOW) {
        for (int t = 0; t < V.w; ++t)
          if (st + t < V.s) dot2_acc(sh, sl, -V.S[r0 * V.w + (int64_t)t * n + r], p[V.nb + st + t]);
      }
    }
    rh[r] = sh;
    rl[r] = sl;
  }
  // a sum of a x over the rows with x = rh + rl: the rh part compensated, the rl part plain
#pragma unroll
  for (int j = 0; j < MM; ++j) {
    if (j < m) {
      float ah = 0.f, al = 0.f;
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < n) {
          const float a = J[j * n + r];
          dot2_acc(ah, al, a, rh[r]);
          al = __fmaf_rn(a, rl[r], al);
        }
      const double d = D[c0 + j];
      g[c0 + j] = ((double)ah + (double)al) - lam * d * d * (double)pj[j];
    }
  }
  if (V.coupled == QRKIT_COUPLED_DENSE) {
    for (int c = 0; c < V.s; ++c) {
      float ah = 0.f, al = 0.f;
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < n) {
          const float a = V.S[(int64_t)c * V.rows + r0 + r];
          dot2_acc(ah, al, a, rh[r]);
          al = __fmaf_rn(a, rl[r], al);
        }
      const double acc = (double)ah + (double)al;
      if (acc != 0.0) atomicAdd(&gS[c], acc);
    }
  } else if (V.coupled == QRKIT_COUPLED_WINDOW) {
    for (int t = 0; t < V.w; ++t) {
      float ah = 0.f, al = 0.f;
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < n) {
          const float a = V.S[r0 * V.w + (int64_t)t * n + r];
          dot2_acc(ah, al, a, rh[r]);
          al = __fmaf_rn(a, rl[r], al);
        }
      const double acc = (double)ah + (double)al;
      if (acc != 0.0 && st + t < V.s) atomicAdd(&gS[st + t - goff], acc);
    }
  }
}

// resid_g_block for blocks of at most NR rows and MM columns, every array in registers.
template <typename T, int NR, int MM>
__device__ __forceinline__ void resid_g_small(const ComposedView<T>& V, const T* b, const T* p, const double* D,
                                              double lam, double* g, double* gS, int64_t goff, int64_t i) {
  if constexpr (sizeof(T) == sizeof(float)) {
    resid_g_small_f32<NR, MM>(V, b, p, D, lam, g, gS, goff, i);
    return;
  }
  const int n = V.n[i], m = V.m[i];
  const int64_t c0 = V.col_off[i], r0 = V.row_off[i];
  const T* J = V.J + V.val_off[i];
  const int64_t st = V.coupled == QRKIT_COUPLED_WINDOW ? V.start[i] : 0;
  double pj[MM], res[NR];
#pragma unroll
  for (int j = 0; j < MM; ++j) pj[j] = j < m ? (double)p[c0 + j] : 0.0;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    double acc = 0.0;
    if (r < n) {
      acc = (double)b[r0 + r];
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (j < m) acc -= (double)J[j * n + r] * pj[j];
      if (V.coupled == QRKIT_COUPLED_DENSE) {
        for (int c = 0; c < V.s; ++c) acc -= (double)V.S[(int64_t)c * V.rows + r0 + r] * (double)p[V.nb + c];
      } else if (V.coupled == QRKIT_COUPLED_WINDOW) {
        for (int t = 0; t < V.w; ++t)
          if (st + t < V.s) acc -= (double)V.S[r0 * V.w + (int64_t)t * n + r] * (double)p[V.nb + st + t];
      }
    }
    res[r] = acc;
  }
#pragma unroll
  for (int j = 0; j < MM; ++j) {
    if (j < m) {
      double acc = 0;
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < n) acc += (double)J[j * n + r] * res[r];
      const double d = D[c0 + j];
      g[c0 + j] = acc - lam * d * d * pj[j];
    }
  }
  if (V.coupled == QRKIT_COUPLED_DENSE) {
    for (int c = 0; c < V.s; ++c) {
      double acc = 0;
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < n) acc += (double)V.S[(int64_t)c * V.rows + r0 + r] * res[r];
      if (acc != 0.0) atomicAdd(&gS[c], acc);
    }
  } else if (V.coupled == QRKIT_COUPLED_WINDOW) {
    for (int t = 0; t < V.w; ++t) {
      double acc = 0;
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < n) acc += (double)V.S[r0 * V.w + (int64_t)t * n + r] * res[r];
      if (acc != 0.0 && st + t < V.s) atomicAdd(&gS[st + t - goff], acc);
    }
  }
}

// Windowed S: the columns the CTA's blocks touch, [lo, hi) with hi = max start + w (uniform
// over the CTA; blocks past K do not count).  The kernels sum into shared memory when the range
// fits (consecutive blocks of one LM problem share its few hundred columns), so a column leaves
// the CTA with one global atomic instead of one per block.
template <typename T>
__device__ __forceinline__ bool window_range(const ComposedView<T>& V, int64_t i, int cap, int64_t& lo, int& width) {
  __shared__ unsigned long long rng[2];
  if (threadIdx.x == 0) {
    rng[0] = ~0ull;
    rng[1] = 0ull;
  }
  __syncthreads();
  unsigned long long mn = ~0ull, mx = 0ull;
  if (i < V.K) mn = mx = (unsigned long long)V.start[i];
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, d));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  }
  if ((threadIdx.x & 31) == 0 && mn != ~0ull) {
    atomicMin(&rng[0], mn);
    atomicMax(&rng[1], mx);
  }
  __syncthreads();
  if (rng[0] == ~0ull) return false;
  lo = (int64_t)rng[0];
  const int64_t w = (int64_t)rng[1] + V.w - lo;
  width = (int)(w < (int64_t)cap ? w : (int64_t)cap);
  return w <= cap;
}

template <typename T, int NA = 0, int MM = 0>
__global__ void resid_g_kernel(ComposedView<T> V, const T* b, const T* p, const double* D,
                               double lam, double* g, double* gS, int win_cols) {
  // dense S: every block adds to all s shared columns; the CTA's sums are gathered in shared
  // memory and leave with one global atomic per column
  extern __shared__ double sgS[];
  const bool cta_sum = V.coupled == QRKIT_COUPLED_DENSE && V.s <= kCtaSumCols;
  if (cta_sum) {
    for (int c = threadIdx.x; c < V.s; c += blockDim.x) sgS[c] = 0.0;
    __syncthreads();
  }
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t lo = 0;
  int width = 0;
  const bool win_sum = V.coupled == QRKIT_COUPLED_WINDOW && win_cols > 0 && window_range(V, i, win_cols, lo, width);
  if (win_sum) {
    for (int c = threadIdx.x; c < width; c += blockDim.x) sgS[c] = 0.0;
    __syncthreads();
  }
  if (i < V.K) {
    if constexpr (NA > 0)
      resid_g_small<T, NA, MM>(V, b, p, D, lam, g, (cta_sum || win_sum) ? sgS : gS, win_sum ? lo : 0, i);
    else
      resid_g_block(V, b, p, D, lam, g, (cta_sum || win_sum) ? sgS : gS, win_sum ? lo : 0, i);
  }
  if (cta_sum) {
    __syncthreads();
    for (int c = threadIdx.x; c < V.s; c += blockDim.x)
      if (sgS[c] != 0.0) atomicAdd(&gS[c], sgS[c]);
  }
  if (win_sum) {
    __syncthreads();
    for (int c = threadIdx.x; c < width; c += blockDim.x)
      if (sgS[c] != 0.0) atomicAdd(&gS[lo + c], sgS[c]);
  }
}

__global__ void gS_damping_kernel(double* gS, const float* pf, const double* pd, const double* D,
                                  int64_t nb, int s, double lam) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  const double pv = pf ? (double)pf[nb + c] : pd[nb + c];
  const double d = D[nb + c];
  gS[c] -= lam * d * d * pv;
}

// h_i = R_i^{-T} g_i per block; then gS -= R12_i^T h_i (dense S: summed per CTA first).
template <typename T>
__device__ __forceinline__ void fwdsub_rt_block(ComposedView<T> V, FactorOut<T> O, const double* g, T* h,
                                                double* gS, int64_t goff, int64_t i) {
  const int n = V.n[i], m = V.m[i];
  const int na = n + (O.damp ? m : 0);
  const int64_t c0 = V.col_off[i];
  const T* F = O.Fa + O.aug_off[i];
  T hv[kMaxCols];
  for (int k = 0; k < m; ++k) {
    T v = (T)g[c0 + k];
    for (int j = 0; j < k; ++j) v -= F[k * na + j] * hv[j];
    hv[k] = v / F[k * na + k];
    h[c0 + k] = hv[k];
  }
  if (V.coupled != QRKIT_COUPLED_NONE) {
    const int64_t st = V.coupled == QRKIT_COUPLED_WINDOW ? V.start[i] : 0;
    for (int t = 0; t < V.w; ++t) {
      if (st + t >= V.s) continue;
      double acc = 0;
      for (int k = 0; k < m; ++k) acc += (double)O.R12[(c0 + k) * (int64_t)V.w + t] * (double)hv[k];
      if (acc != 0.0) atomicAdd(&gS[st + t - goff], -acc);
    }
  }
}

// fwdsub_rt_block for blocks of at most NA augmented rows and MM columns (registers only).
template <typename T, int NA, int MM>
__device__ __forceinline__ void fwdsub_rt_small(const ComposedView<T>& V, const FactorOut<T>& O, const double* g, T* h,
                                                double* gS, int64_t goff, int64_t i) {
  const int n = V.n[i], m = V.m[i];
  const int na = n + (O.damp ? m : 0);
  const int64_t c0 = V.col_off[i];
  const T* F = O.Fa + O.aug_off[i];
  T hv[MM];
#pragma unroll
  for (int k = 0; k < MM; ++k) {
    T v = T(0);
    if (k < m) {
      v = (T)g[c0 + k];
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (j < k) v -= F[k * na + j] * hv[j];
      v = v / F[k * na + k];
      h[c0 + k] = v;
    }
    hv[k] = v;
  }
  if (V.coupled != QRKIT_COUPLED_NONE) {
    const int64_t st = V.coupled == QRKIT_COUPLED_WINDOW ? V.start[i] : 0;
    if constexpr (sizeof(T) == 4 && MM == 1) {
      if (V.coupled == QRKIT_COUPLED_WINDOW && V.w == 8 && m == 1) {
        // one column: R12 row by two 16-byte loads (32-byte aligned), the products in float
        // (h is itself a float correction), each rounded to double once for the sum
        const float4* r4 = reinterpret_cast<const float4*>(O.R12 + c0 * 8);
        const float4 a = r4[0], bq = r4[1];
        const float rv[8] = {a.x, a.y, a.z, a.w, bq.x, bq.y, bq.z, bq.w};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const float prod = rv[t] * hv[0];
          if (prod != 0.f && st + t < V.s) atomicAdd(&gS[st + t - goff], -(double)prod);
        }
        return;
      }
    }
    for (int t = 0; t < V.w; ++t) {
      if (st + t >= V.s) continue;
      double acc = 0;
#pragma unroll
      for (int k = 0; k < MM; ++k)
        if (k < m) acc += (double)O.R12[(c0 + k) * (int64_t)V.w + t] * (double)hv[k];
      if (acc != 0.0) atomicAdd(&gS[st + t - goff], -acc);
    }
  }
}

template <typename T, int NA = 0, int MM = 0>
__global__ void block_fwdsub_rt_kernel(ComposedView<T> V, FactorOut<T> O, const double* g, T* h,
                                       double* gS, int win_cols) {
  extern __shared__ double sgS[];
  const bool cta_sum = V.coupled == QRKIT_COUPLED_DENSE && V.s <= kCtaSumCols;
  if (cta_sum) {
    for (int c = threadIdx.x; c < V.s; c += blockDim.x) sgS[c] = 0.0;
    __syncthreads();
  }
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t lo = 0;
  int width = 0;
  const bool win_sum = V.coupled == QRKIT_COUPLED_WINDOW && win_cols > 0 && window_range(V, i, win_cols, lo, width);
  if (win_sum) {
    for (int c = threadIdx.x; c < width; c += blockDim.x) sgS[c] = 0.0;
    __syncthreads();
  }
  if (i < V.K) {
    if constexpr (NA > 0)
      fwdsub_rt_small<T, NA, MM>(V, O, g, h, (cta_sum || win_sum) ? sgS : gS, win_sum ? lo : 0, i);
    else
      fwdsub_rt_block(V, O, g, h, (cta_sum || win_sum) ? sgS : gS, win_sum ? lo : 0, i);
  }
  if (cta_sum) {
    __syncthreads();
    for (int c = threadIdx.x; c < V.s; c += blockDim.x)
      if (sgS[c] != 0.0) atomicAdd(&gS[c], sgS[c]);
  }
  if (win_sum) {
    __syncthreads();
    for (int c = threadIdx.x; c < width; c += blockDim.x)
      if (sgS[c] != 0.0) atomicAdd(&gS[lo + c], sgS[c]);
  }
}

template <typename T>
__global__ void gS_to_T_kernel(const double* gS, T* out, int s) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < s) out[c] = (T)gS[c];
}

template <typename T>
__global__ void axpy_kernel(T* x, const T* d, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
}

__global__ void widen_kernel(const float* in, double* out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------------------
// Host orchestration.

template <typename T>
static ComposedView<T> view(qrkit_ctx* ctx, const void* J, const void* S) {
  Plan& P = ctx->plan;
  ComposedView<T> V;
  V.K = P.K;
  V.n = (const uint8_t*)P.d_n.ptr;
  V.m = (const uint8_t*)P.d_m.ptr;
  V.val_off = (const int64_t*)P.d_val_off.ptr;
  V.row_off = (const int64_t*)P.d_row_off.ptr;
  V.col_off = (const int64_t*)P.d_col_off.ptr;
  V.start = (const int32_t*)P.d_start.ptr;
  V.coupled = P.s.coupled_kind;
  V.s = (int)P.s.shared_cols;
  V.w = P.s.coupled_kind == QRKIT_COUPLED_DENSE ? (int)P.s.shared_cols : P.s.window;
  V.rows = P.rows;
  V.nb = P.cols;
  V.J = (const T*)J;
  V.S = (const T*)S;
  return V;
}

template <typename T>
static FactorOut<T> fout(qrkit_ctx* ctx) {
  Composed& C = ctx->comp;
  FactorOut<T> O;
  O.damp = C.damp;
  O.lam_half = C.lam_half;
  O.D = (const double*)C.D.ptr;
  O.Fa = (T*)C.Fa.ptr;
  O.tau = (T*)C.tau.ptr;
  O.R12 = (T*)C.R12.ptr;
  O.ctop = (T*)C.ctop.ptr;
  O.aug_off = (const int64_t*)(C.damp ? C.d_aug_off_d.ptr : C.d_aug_off_u.ptr);
  O.red_off = (const int64_t*)(C.damp ? C.d_red_off_d.ptr : C.d_red_off_u.ptr);
  O.X0 = C.levels.empty() ? nullptr : (T*)C.levels[0].X.ptr;
  O.ld0 = C.levels.empty() ? 0 : C.levels[0].ld;
  O.Xw = (T*)C.Xw.ptr;
  O.Xstart = (int64_t*)C.Xstart.ptr;
  O.status = ctx->d_status;
  return O;
}

#define LAUNCH(ctx, ...)                                  \
  do {                                                    \
    __VA_ARGS__;                                          \
    (ctx)->launches += 1;                                 \
    QRKIT_CUDA_TRY(ctx, cudaGetLastError());              \
  } while (0)

// Shape class of a plan's blocks for the per-block kernels: 1 if every augmented block is at
// most 3 x 1, 2 if at most 6 x 2, else 0 (the general kernels with runtime loops).
int small_class(const Plan& P, bool damp) {
  const int na = P.max_n + (damp ? P.max_m : 0);
  if (P.max_m == 1 && na <= 3) return 1;
  if (P.max_m <= 2 && na <= 6) return 2;
  return 0;
}
// A per-block kernel template KERNEL<T, NA, MM> launched in the instantiation of the class.
#define LAUNCH_SHAPED(ctx, cls, KERNEL, grid, threads, smem, stream, ...)                      \
  do {                                                                                         \
    if ((cls) == 1) LAUNCH(ctx, (KERNEL<T, 3, 1><<<grid, threads, smem, stream>>>(__VA_ARGS__))); \
    else if ((cls) == 2) LAUNCH(ctx, (KERNEL<T, 6, 2><<<grid, threads, smem, stream>>>(__VA_ARGS__))); \
    else LAUNCH(ctx, (KERNEL<T><<<grid, threads, smem, stream>>>(__VA_ARGS__)));                \
  } while (0)

// D = column norms of J (Sec. 5.2), zero -> 1, in double; C.sq is the scratch.
template <typename T>
static qrkit_status norms_typed(qrkit_ctx* ctx, const ComposedView<T>& V, double* D) {
  Plan& P = ctx->plan;
  Composed& C = ctx->comp;
  cudaStream_t st = ctx->stream;
  const int64_t N = P.cols + P.s.shared_cols;
  qrkit_status rc;
  // dense S: the chunk sums of pass 1 follow the N column sums in the same scratch
  const int64_t nchunk = V.coupled == QRKIT_COUPLED_DENSE ? std::max<int64_t>(1, (V.rows + kNormRows - 1) / kNormRows) : 0;
  const size_t sq_bytes = (size_t)(N + nchunk * (V.coupled == QRKIT_COUPLED_DENSE ? V.s : 0)) * sizeof(double);
  if ((rc = ensure(ctx, C.sq, sq_bytes, "column sums")) != QRKIT_OK) return rc;
  double* sq = (double*)C.sq.ptr;
  QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(sq, 0, (size_t)N * sizeof(double), st));
  LAUNCH(ctx, colnorm_blocks_kernel<T><<<blocks_for(P.K, 128), 128, 0, st>>>(V, sq));
  if (V.coupled == QRKIT_COUPLED_DENSE) {
    if (nchunk > (int64_t)INT32_MAX) return fail(ctx, QRKIT_EUNSUPPORTED, "too many rows for the column norms");
    const dim3 grid((unsigned)nchunk, (unsigned)std::min<int64_t>(V.s, 65535));
    LAUNCH(ctx, colnorm_dense_part_kernel<T><<<grid, kNormThreads, 0, st>>>(V, sq + N, nchunk));
    LAUNCH(ctx, colnorm_dense_sum_kernel<<<blocks_for(V.s, 128), 128, 0, st>>>(sq + N, nchunk, V.s, sq + V.nb));
  } else if (V.coupled == QRKIT_COUPLED_WINDOW)
    LAUNCH(ctx, colnorm_window_kernel<T><<<blocks_for(P.K, 128), 128, 0, st>>>(V, sq));
  LAUNCH(ctx, finalize_norms_kernel<<<blocks_for(N, 256), 256, 0, st>>>(sq, D, N));
  return QRKIT_OK;
}

// Column-panel TSQR of a float dense reduced block (s a multiple of 32 above 32).  Panel j
// (columns c0 = 32 j ..): its levels are factored tile by tile (R rows up; the top level's into
// R_S), and after each level the tiles' Q^T is applied to the panel's trailing columns on the
// tensor cores, whose rows move up with the R rows or down into the next panel's first level.
// Narrow panels keep the column-by-column part of the work (the tile QR) small: it grows with the
// panel width, while the trailing updates do the rest of the arithmetic.
static qrkit_status factor_panels(qrkit_ctx* ctx, int s) {
  Composed& C = ctx->comp;
  cudaStream_t st = ctx->stream;
  float* Rs = (float*)C.Rs.ptr;
  const int np = 1 + (int)C.panels.size();
  for (int j = 0; j < np; ++j) {
    std::vector<TsqrLevel>& LV = j == 0 ? C.levels : C.panels[j - 1].levels;
    const int c0 = j * kPanelCols;
    const int pw = std::min(kPanelCols, s - c0);
    const int n = s - c0 - pw;   // trailing columns
    if (pw != kPanelCols) return fail(ctx, QRKIT_EINVAL, "column panels: s must be a multiple of 32");
    for (size_t l = 0; l < LV.size(); ++l) {
      TsqrLevel& L = LV[l];
      const bool top = l + 1 == LV.size();
      float* X = (float*)L.X.ptr;
      float* Xn = top ? Rs + (int64_t)c0 * s + c0 : (float*)LV[l + 1].X.ptr;
      const int64_t ldn = top ? s : LV[l + 1].ld;
      qrkit_status rc = tsqr_panel_tile(ctx, X, L.ld, L.M, (float*)L.tau.ptr, Xn, ldn, L.tiles,
                                        n > 0 ? (float*)L.T.ptr : nullptr);
      if (rc != QRKIT_OK) return rc;
      if (n > 0) {
        float* upp = top ? Rs + (int64_t)(c0 + pw) * s + c0 : (float*)LV[l + 1].X.ptr + (int64_t)pw * LV[l + 1].ld;
        const int64_t ldu = top ? s : LV[l + 1].ld;
        TsqrLevel& N0 = C.panels[j].levels[0];
        rc = tsqr_panel_apply(ctx, X, L.ld, L.M, pw, (const float*)L.T.ptr, n, upp, ldu, (float*)N0.X.ptr, N0.ld,
                              L.down0, L.tiles);
        if (rc != QRKIT_OK) return rc;
      }
    }
  }
  return QRKIT_OK;
}

template <typename T>
static qrkit_status factor_typed(qrkit_ctx* ctx, const void* J, const void* S, const void* Dext,
                                 double lambda, bool dext_double = false) {
  Plan& P = ctx->plan;
  Composed& C = ctx->comp;
  cudaStream_t st = ctx->stream;
  const int64_t N = P.cols + P.s.shared_cols;
  qrkit_status rc;
  if ((rc = ensure(ctx, C.D, (size_t)N * sizeof(double), "D")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.sq, (size_t)N * sizeof(double), "column sums")) != QRKIT_OK) return rc;
  C.damp = lambda > 0.0;
  C.lam = lambda;
  C.lam_half = sqrt(lambda);
  if ((rc = composed_layout(ctx, sizeof(T))) != QRKIT_OK) return rc;
  ComposedView<T> V = view<T>(ctx, J, S);
  // D: caller's (copied to double) or column norms of J
  if (Dext) {
    if (sizeof(T) == sizeof(double) || dext_double) {
      QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(C.D.ptr, Dext, (size_t)N * sizeof(double),
                                          cudaMemcpyDeviceToDevice, st));
    } else {
      rc = widen_to_double(ctx, (const float*)Dext, (double*)C.D.ptr, N);
      if (rc != QRKIT_OK) return rc;
    }
  } else if ((rc = norms_typed<T>(ctx, V, (double*)C.D.ptr)) != QRKIT_OK) {
    return rc;
  }
  FactorOut<T> O = fout<T>(ctx);
  // the small-block kernels when every block fits them (e.g. 2 x 1 blocks of curve fits)
  const int cls = small_class(P, O.damp);
  if (cls == 1)
    LAUNCH(ctx, (block_factor_small_kernel<T, 3, 1><<<blocks_for(P.K, 128), 128, 0, st>>>(V, O)));
  else if (cls == 2)
    LAUNCH(ctx, (block_factor_small_kernel<T, 6, 2><<<blocks_for(P.K, 128), 128, 0, st>>>(V, O)));
  else
    LAUNCH(ctx, block_factor_kernel<T><<<blocks_for(P.K, 64), 64, 0, st>>>(V, O));
  if (V.coupled == QRKIT_COUPLED_WINDOW) {
    // P_r of the reduced block: its rows sorted by leading column per segment (Sec. 4.3)
    rc = reduced_row_sort(ctx, C.sort, (int64_t)P.seg_cols.size(), C.sort_hist_entries,
                          (const int64_t*)C.Xstart.ptr, C.Xw.ptr, V.w, (int*)C.hist.ptr,
                          (int64_t*)C.spos.ptr, (int64_t*)C.order.ptr, (int64_t*)C.Xstart_s.ptr, C.Xw_s.ptr);
    if (rc != QRKIT_OK) return rc;
  }
  if (V.coupled == QRKIT_COUPLED_DENSE) {
    const int s = V.s;
    if (C.damp)
      LAUNCH(ctx, reduced_damping_kernel<T><<<blocks_for((int64_t)s * s, 256), 256, 0, st>>>(
                      (T*)C.levels[0].X.ptr, C.levels[0].ld, C.red_rows, s, (const double*)C.D.ptr,
                      P.cols, C.lam_half));
    if (!C.panels.empty()) return factor_panels(ctx, s);
    for (size_t l = 0; l < C.levels.size(); ++l) {
      TsqrLevel& L = C.levels[l];
      T* Xn = l + 1 < C.levels.size() ? (T*)C.levels[l + 1].X.ptr : nullptr;
      const int64_t ldn = l + 1 < C.levels.size() ? C.levels[l + 1].ld : 0;
      const size_t smem = ((size_t)C.tile_rows * s + 64) * sizeof(T);
      auto k = tsqr_tile_kernel<T>;
      QRKIT_CUDA_TRY(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      LAUNCH(ctx, k<<<(unsigned)L.tiles, kTileThreads, smem, st>>>((T*)L.X.ptr, L.ld, L.M, s, C.tile_rows,
                                                                  (T*)L.tau.ptr, Xn, ldn, ctx->d_status));
    }
  }
  return QRKIT_OK;
}

template <typename T>
static qrkit_status solve_typed(qrkit_ctx* ctx, const void* J, const void* S, const void* b, void* p,
                                int refine_steps, bool qt_only, void* qtb_out) {
  Plan& P = ctx->plan;
  Composed& C = ctx->comp;
  cudaStream_t st = ctx->stream;
  ComposedView<T> V = view<T>(ctx, J, S);
  FactorOut<T> O = fout<T>(ctx);
  const int s = V.s;
  const int64_t nb = P.cols;
  T* x = (T*)p;
  // Q^T [b; 0]
  T* rhs0 = (V.coupled == QRKIT_COUPLED_DENSE) ? (T*)C.levels[0].rhs.ptr
             : (V.coupled == QRKIT_COUPLED_WINDOW ? (T*)C.rhs_red.ptr : nullptr);
  LAUNCH_SHAPED(ctx, small_class(P, O.damp), block_apply_qt_kernel, blocks_for(P.K, 64), 64, 0, st, V, O, (const T*)b,
                rhs0);
  if (V.coupled == QRKIT_COUPLED_DENSE) {
    if (C.damp)
      QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(rhs0 + C.red_rows, 0, (size_t)s * sizeof(T), st));
    // Q^T of every panel's levels: the top rows of a level go up (the last level's into c_S),
    // the others, with column panels, into the next panel's first level
    const int np = 1 + (int)C.panels.size();
    for (int j = 0; j < np; ++j) {
      std::vector<TsqrLevel>& LV = j == 0 ? C.levels : C.panels[j - 1].levels;
      const int c0 = j == 0 ? 0 : C.panels[j - 1].c0;
      const int pw = j == 0 ? C.panel0_w : C.panels[j - 1].pw;
      T* down = j + 1 < np ? (T*)C.panels[j].levels[0].rhs.ptr : nullptr;
      for (size_t l = 0; l < LV.size(); ++l) {
        TsqrLevel& L = LV[l];
        const bool top = l + 1 == LV.size();
        T* rn = !top ? (T*)LV[l + 1].rhs.ptr : (np > 1 ? (T*)C.cs.ptr + c0 : nullptr);
        LAUNCH(ctx, tsqr_apply_qt_kernel<T><<<(unsigned)L.tiles, kTileThreads, 0, st>>>(
                        (const T*)L.X.ptr, L.ld, L.M, pw, C.tile_rows, (const T*)L.tau.ptr, (T*)L.rhs.ptr, rn, down,
                        L.down0));
      }
    }
  }
  if (V.coupled == QRKIT_COUPLED_WINDOW && qt_only)
    return fail(ctx, QRKIT_EUNSUPPORTED, "Q^T b is not kept for windowed structures (use qrkit_solve)");
  if (qt_only) {
    // Q^T b reported as [c_blocks (sum m_i); c_S (s)]
    T* out = (T*)qtb_out;
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(out, O.ctop, (size_t)nb * sizeof(T), cudaMemcpyDeviceToDevice, st));
    if (s > 0)
      QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(out + nb, C.panels.empty() ? C.levels.back().rhs.ptr : C.cs.ptr,
                                          (size_t)s * sizeof(T), cudaMemcpyDeviceToDevice, st));
    return QRKIT_OK;
  }
  // R_S and c_S: the top level's rows, or the panels' R rows gathered in Rs and cs
  const TsqrLevel* top = C.levels.empty() ? nullptr : &C.levels.back();
  const bool pan = !C.panels.empty();
  const T* RS = pan ? (const T*)C.Rs.ptr : (top ? (const T*)top->X.ptr : nullptr);
  const int64_t ldRS = pan ? s : (top ? top->ld : 0);
  if (V.coupled == QRKIT_COUPLED_DENSE) {
    LAUNCH(ctx, dense_backsub_kernel<T><<<1, tri_threads(s), 0, st>>>(
                    RS, ldRS, s, pan ? (const T*)C.cs.ptr : (const T*)top->rhs.ptr, x + nb, 0, ctx->d_status));
  } else if (V.coupled == QRKIT_COUPLED_WINDOW) {
    // reduced banded block of every segment (Sec. 4.4), rows in P_r order, the shared
    // columns' damping rows interleaved
    qrkit_status rc = reduced_rhs_sort(ctx, (const int64_t*)C.spos.ptr, C.rhs_red.ptr, C.rhs_s.ptr, C.red_rows);
    if (rc != QRKIT_OK) return rc;
    if (C.cr)
      rc = cr_solve(ctx, *C.cr, (const int64_t*)C.Xstart_s.ptr, 1, V.w, C.Xw_s.ptr, C.rhs_s.ptr, O.D + nb,
                    C.damp ? C.lam : 0.0, x + nb, (double*)C.res2.ptr);
    else
      rc = banded_explicit_solve(ctx, (int64_t)P.seg_cols.size(), (const int64_t*)C.seg_inst.ptr, C.Xw_s.ptr,
                                 (const int64_t*)C.Xstart_s.ptr, C.rhs_s.ptr, V.w, O.D + nb,
                                 C.damp ? C.lam : 0.0, C.RwS.ptr, C.cS.ptr, x + nb, (double*)C.res2.ptr);
    if (rc != QRKIT_OK) return rc;
  }
  LAUNCH_SHAPED(ctx, small_class(P, O.damp), block_backsub_kernel, blocks_for(P.K, 64), 64, 0, st, V, O, O.ctop,
                s ? x + nb : nullptr, x, 0);
  // refinement (extended-precision residual, corrections through R only)
  for (int it = 0; it < refine_steps; ++it) {
    const int64_t N = nb + s;
    qrkit_status rc;
    if ((rc = ensure(ctx, C.g, (size_t)N * sizeof(double), "refinement g")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.h, (size_t)N * sizeof(T), "refinement h")) != QRKIT_OK) return rc;
    double* g = (double*)C.g.ptr;
    T* h = (T*)C.h.ptr;
    double* gS = g + nb;
    if (s > 0) QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(gS, 0, (size_t)s * sizeof(double), st));
    // dense S: all s columns per CTA; windowed S: the CTA's column range (up to kWinSumCols),
    // with larger CTAs so that more blocks share a column sum
    const bool win = V.coupled == QRKIT_COUPLED_WINDOW;
    const int rthreads = win ? 256 : 64;
    const size_t sum_smem = (V.coupled == QRKIT_COUPLED_DENSE && s <= kCtaSumCols) ? (size_t)s * sizeof(double)
                            : win ? (size_t)kWinSumCols * sizeof(double) : 0;
    const int win_cols = win ? kWinSumCols : 0;
    LAUNCH_SHAPED(ctx, small_class(P, O.damp), resid_g_kernel, blocks_for(P.K, rthreads), rthreads, sum_smem, st, V,
                  (const T*)b, x, O.D, C.lam, g, gS, win_cols);
    if (s > 0)
      LAUNCH(ctx, gS_damping_kernel<<<blocks_for(s, 128), 128, 0, st>>>(
                      gS, sizeof(T) == 4 ? (const float*)x : nullptr,
                      sizeof(T) == 8 ? (const double*)x : nullptr, O.D, nb, s, C.lam));
    LAUNCH_SHAPED(ctx, small_class(P, O.damp), block_fwdsub_rt_kernel, blocks_for(P.K, rthreads), rthreads, sum_smem,
                  st, V, O, g, h, gS, win_cols);
    if (V.coupled == QRKIT_COUPLED_WINDOW && C.cr) {
      // dp_S = R_S^{-1} R_S^{-T} (g_S - R12^T h_B) with the parallel banded factor
      qrkit_status rc = cr_normal_solve(ctx, *C.cr, gS, h + nb);
      if (rc != QRKIT_OK) return rc;
      LAUNCH(ctx, axpy_kernel<T><<<blocks_for(s, 128), 128, 0, st>>>(x + nb, h + nb, s));
    } else if (V.coupled == QRKIT_COUPLED_WINDOW) {
      // h_S = R_S^{-T} (g_S - R12^T h_B), then dp_S = R_S^{-1} h_S, both banded
      LAUNCH(ctx, gS_to_T_kernel<T><<<blocks_for(s, 128), 128, 0, st>>>(gS, h + nb, s));
      const int64_t nseg = (int64_t)P.seg_cols.size();
      const int64_t* inst = (const int64_t*)C.seg_inst.ptr;
      qrkit_status rc = banded_tri_solve(ctx, nseg, inst, C.RwS.ptr, V.w, h + nb, true);
      if (rc != QRKIT_OK) return rc;
      rc = banded_tri_solve(ctx, nseg, inst, C.RwS.ptr, V.w, h + nb, false);
      if (rc != QRKIT_OK) return rc;
      LAUNCH(ctx, axpy_kernel<T><<<blocks_for(s, 128), 128, 0, st>>>(x + nb, h + nb, s));
    }
    if (V.coupled == QRKIT_COUPLED_DENSE) {
      // h_S = R_S^{-T} (g_S - R12^T h_B), then dp_S = R_S^{-1} h_S in place
      LAUNCH(ctx, dense_fwdsub_rt_kernel<T><<<1, tri_threads(s), 0, st>>>(RS, ldRS, s, gS, h + nb));
      LAUNCH(ctx, dense_backsub_kernel<T><<<1, tri_threads(s), 0, st>>>(RS, ldRS, s, h + nb, h + nb, 0,
                                                                         ctx->d_status));
      LAUNCH(ctx, axpy_kernel<T><<<blocks_for(s, 128), 128, 0, st>>>(x + nb, h + nb, s));
    }
    // dp_B = R_B^{-1} (h_B - R12 dp_S), accumulated into p
    LAUNCH_SHAPED(ctx, small_class(P, O.damp), block_backsub_kernel, blocks_for(P.K, 64), 64, 0, st, V, O, h,
                  s ? h + nb : nullptr, x, 1);
  }
  return QRKIT_OK;
}

qrkit_status composed_factor(qrkit_ctx* ctx, const void* J, const void* S, const void* D, double lambda) {
  if (ctx->precision == QRKIT_FP64) return factor_typed<double>(ctx, J, S, D, lambda);
  return factor_typed<float>(ctx, J, S, D, lambda);
}

template <typename T>
ComposedView<T> composed_view(qrkit_ctx* ctx, const void* J, const void* S) {
  return view<T>(ctx, J, S);
}
template ComposedView<float> composed_view<float>(qrkit_ctx*, const void*, const void*);
template ComposedView<double> composed_view<double>(qrkit_ctx*, const void*, const void*);

qrkit_status composed_column_norms(qrkit_ctx* ctx, const void* J, const void* S, double* D) {
  if (ctx->precision == QRKIT_FP64) return norms_typed<double>(ctx, view<double>(ctx, J, S), D);
  return norms_typed<float>(ctx, view<float>(ctx, J, S), D);
}

qrkit_status composed_factor_scaled(qrkit_ctx* ctx, const void* J, const void* S, const double* E) {
  if (ctx->precision == QRKIT_FP64) return factor_typed<double>(ctx, J, S, E, 1.0, true);
  return factor_typed<float>(ctx, J, S, E, 1.0, true);
}

qrkit_status composed_solve(qrkit_ctx* ctx, const void* J, const void* S, const void* b, void* p,
                            int refine_steps) {
  if (ctx->precision == QRKIT_FP64) return solve_typed<double>(ctx, J, S, b, p, refine_steps, false, nullptr);
  const int steps = ctx->precision == QRKIT_FP32 ? 0 : refine_steps;
  return solve_typed<float>(ctx, J, S, b, p, steps, false, nullptr);
}

qrkit_status composed_apply_qt(qrkit_ctx* ctx, const void* b, void* qtb) {
  if (ctx->precision == QRKIT_FP64) return solve_typed<double>(ctx, nullptr, nullptr, b, nullptr, 0, true, qtb);
  return solve_typed<float>(ctx, nullptr, nullptr, b, nullptr, 0, true, qtb);
}

}  // namespace qrkit

namespace qrkit {

static qrkit_status upload_i64(qrkit_ctx* ctx, DevBuf& buf, const std::vector<int64_t>& v, const char* what) {
  qrkit_status rc = ensure(ctx, buf, v.size() * sizeof(int64_t), what);
  if (rc != QRKIT_OK) return rc;
  QRKIT_CUDA_TRY(ctx, cudaMemcpy(buf.ptr, v.data(), v.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  return QRKIT_OK;
}

qrkit_status widen_to_double(qrkit_ctx* ctx, const float* in, double* out, int64_t n) {
  widen_kernel<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(in, out, n);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

static void release_levels(std::vector<TsqrLevel>& LV) {
  for (auto& L : LV) { release(L.X); release(L.tau); release(L.rhs); release(L.T); }
  LV.clear();
}

void release_composed(Composed& C) {
  release(C.D); release(C.sq); release(C.Fa); release(C.tau); release(C.R12); release(C.ctop);
  release(C.g); release(C.h);
  release(C.Xw); release(C.Xstart); release(C.rhs_red); release(C.RwS); release(C.cS);
  release(C.res2); release(C.meta); release(C.dense_ws);
  release(C.sort_tab); release(C.hist); release(C.spos); release(C.order); release(C.Xw_s);
  release(C.Xstart_s); release(C.rhs_s); release(C.seg_inst);
  release_cr(C.cr);
  release(C.nrm_D); release(C.nrm_L); release(C.nrm_W); release(C.nrm_y); release(C.nrm_As);
  release(C.nrm_rs); release(C.nrm_seg);
  release(C.d_aug_off_d); release(C.d_aug_off_u); release(C.d_red_off_d); release(C.d_red_off_u);
  release_levels(C.levels);
  for (auto& Pn : C.panels) release_levels(Pn.levels);
  release(C.Rs); release(C.cs);
  C = Composed();
}

// Reduced-row offsets per block (host) with / without damping rows.
static std::vector<int64_t> reduced_offsets(const Plan& P, bool damp) {
  std::vector<int64_t> r(P.K + 1, 0);
  for (int64_t i = 0; i < P.K; ++i) r[i + 1] = r[i] + (damp ? P.n[i] : P.n[i] - P.m[i]);
  return r;
}

// Offsets of the augmented blocks for both damping states, the factor buffers, and the
// TSQR level geometry of the dense reduced block.
qrkit_status composed_layout(qrkit_ctx* ctx, size_t elem) {
  Plan& P = ctx->plan;
  Composed& C = ctx->comp;
  qrkit_status rc;
  if (!C.d_aug_off_d.ptr) {
    std::vector<int64_t> ad(P.K + 1), au(P.K + 1), rd(P.K + 1), ru(P.K + 1);
    ad[0] = au[0] = rd[0] = ru[0] = 0;
    for (int64_t i = 0; i < P.K; ++i) {
      const int64_t n = P.n[i], m = P.m[i];
      ad[i + 1] = ad[i] + (n + m) * m;
      au[i + 1] = au[i] + n * m;
      rd[i + 1] = rd[i] + n;
      ru[i + 1] = ru[i] + (n - m);
    }
    C.aug_values_d = ad[P.K]; C.aug_values_u = au[P.K];
    C.red_rows_d = rd[P.K]; C.red_rows_u = ru[P.K];
    if ((rc = upload_i64(ctx, C.d_aug_off_d, ad, "aug offsets")) != QRKIT_OK) return rc;
    if ((rc = upload_i64(ctx, C.d_aug_off_u, au, "aug offsets")) != QRKIT_OK) return rc;
    if ((rc = upload_i64(ctx, C.d_red_off_d, rd, "reduced offsets")) != QRKIT_OK) return rc;
    if ((rc = upload_i64(ctx, C.d_red_off_u, ru, "reduced offsets")) != QRKIT_OK) return rc;
  }
  if (C.damp && P.first_tall_aug >= 0)
    return fail(ctx, QRKIT_EUNSUPPORTED, "block " + std::to_string(P.first_tall_aug) +
                ": with damping rows the augmented block exceeds 16 rows");
  if (!C.damp && P.first_wide >= 0)
    return fail(ctx, QRKIT_EINVAL, "block " + std::to_string(P.first_wide) +
                " has fewer rows than columns and lambda = 0");
  C.red_rows = C.damp ? C.red_rows_d : C.red_rows_u;
  const int64_t aug = C.damp ? C.aug_values_d : C.aug_values_u;
  {
    const int64_t N = P.cols + P.s.shared_cols;
    if ((rc = ensure(ctx, C.g, (size_t)N * sizeof(double), "refinement g")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.h, (size_t)N * elem, "refinement h")) != QRKIT_OK) return rc;
  }
  const int s = (int)P.s.shared_cols;
  const int w = P.s.coupled_kind == QRKIT_COUPLED_DENSE ? s : P.s.window;
  if ((rc = ensure(ctx, C.Fa, (size_t)aug * elem, "factor")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.tau, (size_t)P.cols * elem, "tau")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.ctop, (size_t)P.cols * elem, "c")) != QRKIT_OK) return rc;
  if (P.s.coupled_kind != QRKIT_COUPLED_NONE)
    if ((rc = ensure(ctx, C.R12, (size_t)P.cols * w * elem, "R12")) != QRKIT_OK) return rc;
  if (P.s.coupled_kind == QRKIT_COUPLED_WINDOW) {
    // the reduced rows form a banded matrix (rows sorted by window start); its QR runs with
    // the right-hand side in qrkit_solve (the banded solver does not keep Q)
    const int64_t Mr = C.red_rows > 0 ? C.red_rows : 1;
    if ((rc = ensure(ctx, C.Xw, (size_t)Mr * w * elem, "reduced rows")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.Xstart, (size_t)Mr * sizeof(int64_t), "reduced row starts")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.rhs_red, (size_t)Mr * elem, "reduced rhs")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.RwS, (size_t)s * w * elem, "reduced R")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.cS, (size_t)s * elem, "reduced c")) != QRKIT_OK) return rc;
    const int64_t nseg = (int64_t)P.seg_cols.size();
    if ((rc = ensure(ctx, C.res2, sizeof(double) * nseg, "reduced residual")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.spos, (size_t)Mr * sizeof(int64_t), "reduced row order")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.order, (size_t)Mr * sizeof(int64_t), "reduced row order")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.Xw_s, (size_t)Mr * w * elem, "sorted reduced rows")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.Xstart_s, (size_t)Mr * sizeof(int64_t), "sorted row starts")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.rhs_s, (size_t)Mr * elem, "sorted reduced rhs")) != QRKIT_OK) return rc;
    if (C.sort_damp != (C.damp ? 1 : 0)) {
      // chunk tables of the device row sort and the segments' banded instances (host, once
      // per damping state: the reduced rows per block differ with and without damping rows)
      const std::vector<int64_t> ro = reduced_offsets(P, C.damp);
      std::vector<int64_t> c_row0, c_rows, c_hoff, c_col0, c_cols, c_out0, seg_chunk0(nseg + 1, 0);
      std::vector<int64_t> inst(4 * nseg);
      int64_t hoff = 0;
      for (int64_t k = 0; k < nseg; ++k) {
        const int64_t r0 = ro[P.seg_blk0[k]], r1 = ro[P.seg_blk0[k + 1]];
        const int64_t rows = r1 - r0;
        if (rows >= ((int64_t)1 << 31))
          return fail(ctx, QRKIT_EUNSUPPORTED, "a segment has more than 2^31 reduced rows");
        int64_t per = std::max<int64_t>(2048, (rows + 255) / 256);
        seg_chunk0[k] = (int64_t)c_row0.size();
        for (int64_t q = r0; q < r1; q += per) {
          c_row0.push_back(q);
          c_rows.push_back(std::min(per, r1 - q));
          c_hoff.push_back(hoff);
          c_col0.push_back(P.seg_col0[k]);
          c_cols.push_back(P.seg_cols[k]);
          c_out0.push_back(r0);
          hoff += P.seg_cols[k];
        }
        inst[k] = P.seg_cols[k];
        inst[nseg + k] = P.seg_col0[k];
        inst[2 * nseg + k] = r0;
        inst[3 * nseg + k] = rows;
      }
      seg_chunk0[nseg] = (int64_t)c_row0.size();
      if (hoff > ((int64_t)1 << 28))
        return fail(ctx, QRKIT_EUNSUPPORTED, "segments too wide for the device row sort");
      const int64_t nc = (int64_t)c_row0.size();
      std::vector<int64_t> tab;
      for (auto* v : {&c_row0, &c_rows, &c_hoff, &c_col0, &c_cols, &c_out0}) tab.insert(tab.end(), v->begin(), v->end());
      tab.insert(tab.end(), seg_chunk0.begin(), seg_chunk0.end());
      if ((rc = upload_i64(ctx, C.sort_tab, tab, "row sort tables")) != QRKIT_OK) return rc;
      if ((rc = upload_i64(ctx, C.seg_inst, inst, "segment instances")) != QRKIT_OK) return rc;
      if (w <= 8) {
        std::vector<int64_t> ic(inst.begin(), inst.begin() + nseg), i0(inst.begin() + nseg, inst.begin() + 2 * nseg),
            r0v(inst.begin() + 2 * nseg, inst.begin() + 3 * nseg), rv(inst.begin() + 3 * nseg, inst.end());
        if ((rc = cr_build(ctx, C.cr, ic, i0, r0v, rv)) != QRKIT_OK) return rc;
      }
      // histograms, then one bin total per shared column (the scan's second pass)
      if ((rc = ensure(ctx, C.hist, (size_t)std::max<int64_t>(hoff + P.s.shared_cols, 1) * sizeof(int),
                       "row sort histograms")) != QRKIT_OK)
        return rc;
      const int64_t* t = (const int64_t*)C.sort_tab.ptr;
      C.sort.num_chunks = nc;
      C.sort.chunk_row0 = t;
      C.sort.chunk_rows = t + nc;
      C.sort.chunk_hoff = t + 2 * nc;
      C.sort.chunk_col0 = t + 3 * nc;
      C.sort.chunk_cols = t + 4 * nc;
      C.sort.chunk_out0 = t + 5 * nc;
      C.sort.seg_chunk0 = t + 6 * nc;
      C.sort_hist_entries = hoff;
      C.sort_damp = C.damp ? 1 : 0;
    }
  }
  if (P.s.coupled_kind == QRKIT_COUPLED_DENSE) {
    // float, s a multiple of 32 above 32: column panels of kPanelCols, each a TSQR of its own,
    // their trailing updates on the tensor cores; otherwise one TSQR of CUDA-core tiles (s <= 64)
    const bool panels = elem == sizeof(float) && s > kPanelCols && s <= kMaxDenseS && s % 32 == 0;
    if (s > 64 && !panels)
      return fail(ctx, QRKIT_EUNSUPPORTED,
                  "dense shared block: s <= 64, or (float) s a multiple of 32 up to 512");
    const int64_t M0 = C.red_rows + (C.damp ? s : 0);
    if (M0 < s) return fail(ctx, QRKIT_EINVAL, "reduced shared block has fewer rows than columns");
    C.tile_rows = 256;
    // the TSQR levels of a panel of pw columns over M rows, w columns wide (panel + trailing);
    // each level's leading dimension is padded to 16 bytes, and the rows that leave a panel
    // (all but its R rows) are laid out level by level, tile by tile, for the next panel
    auto build_levels = [&](std::vector<TsqrLevel>& LV, int64_t M, int pw, int w, bool need_T) -> qrkit_status {
      std::vector<int64_t> Ms;
      while (true) {
        Ms.push_back(M);
        const int64_t tiles = (M + C.tile_rows - 1) / C.tile_rows;
        if (tiles <= 1) break;
        const int64_t last = M - (tiles - 1) * C.tile_rows;
        M = (tiles - 1) * pw + std::min<int64_t>(last, pw);
      }
      if (LV.size() != Ms.size()) {
        release_levels(LV);
        LV.assign(Ms.size(), TsqrLevel());
      }
      int64_t down = 0;
      qrkit_status rc2;
      for (size_t l = 0; l < Ms.size(); ++l) {
        TsqrLevel& L = LV[l];
        L.M = Ms[l];
        L.ld = (L.M + 3) & ~int64_t(3);
        L.tiles = (L.M + C.tile_rows - 1) / C.tile_rows;
        L.down0 = down;
        down += L.M - (l + 1 < Ms.size() ? Ms[l + 1] : (int64_t)pw);
        if ((rc2 = ensure(ctx, L.X, (size_t)L.ld * w * elem, "reduced block")) != QRKIT_OK) return rc2;
        if ((rc2 = ensure(ctx, L.tau, (size_t)L.tiles * pw * elem, "reduced tau")) != QRKIT_OK) return rc2;
        if ((rc2 = ensure(ctx, L.rhs, (size_t)L.ld * elem, "reduced rhs")) != QRKIT_OK) return rc2;
        if (need_T && (rc2 = ensure(ctx, L.T, (size_t)L.tiles * pw * 32 * elem, "reduced T")) != QRKIT_OK)
          return rc2;
      }
      return QRKIT_OK;
    };
    C.panel0_w = panels ? kPanelCols : s;
    if ((rc = build_levels(C.levels, M0, C.panel0_w, s, panels)) != QRKIT_OK) return rc;
    if (panels) {
      const int np = (s + kPanelCols - 1) / kPanelCols;
      if ((int)C.panels.size() != np - 1) {
        for (auto& Pn : C.panels) release_levels(Pn.levels);
        C.panels.assign(np - 1, TsqrPanel());
      }
      for (int j = 1; j < np; ++j) {
        TsqrPanel& Pn = C.panels[j - 1];
        Pn.c0 = j * kPanelCols;
        Pn.pw = std::min(kPanelCols, s - Pn.c0);
        Pn.w = s - Pn.c0;
        if ((rc = build_levels(Pn.levels, M0 - Pn.c0, Pn.pw, Pn.w, j + 1 < np)) != QRKIT_OK) return rc;
      }
      if ((rc = ensure(ctx, C.Rs, (size_t)s * s * elem, "R_S")) != QRKIT_OK) return rc;
      if ((rc = ensure(ctx, C.cs, (size_t)s * elem, "R_S rhs")) != QRKIT_OK) return rc;
    } else {
      for (auto& Pn : C.panels) release_levels(Pn.levels);
      C.panels.clear();
    }
  } else {
    release_levels(C.levels);
    for (auto& Pn : C.panels) release_levels(Pn.levels);
    C.panels.clear();
  }
  return QRKIT_OK;
}

template <typename T>
static qrkit_status solve_r_typed(qrkit_ctx* ctx, const void* qtb, void* p) {
  Plan& P = ctx->plan;
  if (P.s.coupled_kind == QRKIT_COUPLED_WINDOW)
    return fail(ctx, QRKIT_EUNSUPPORTED, "R of a windowed structure is formed in qrkit_solve");
  Composed& C = ctx->comp;
  cudaStream_t st = ctx->stream;
  ComposedView<T> V = view<T>(ctx, nullptr, nullptr);
  FactorOut<T> O = fout<T>(ctx);
  const int s = V.s;
  const T* c = (const T*)qtb;
  T* x = (T*)p;
  if (V.coupled == QRKIT_COUPLED_DENSE) {
    const TsqrLevel& top = C.levels.back();
    const bool pan = !C.panels.empty();
    LAUNCH(ctx, dense_backsub_kernel<T><<<1, tri_threads(s), 0, st>>>(
                    pan ? (const T*)C.Rs.ptr : (const T*)top.X.ptr, pan ? s : top.ld, s, c + P.cols, x + P.cols, 0,
                    ctx->d_status));
  }
  LAUNCH(ctx, block_backsub_kernel<T><<<blocks_for(P.K, 64), 64, 0, st>>>(V, O, c, s ? x + P.cols : nullptr, x, 0));
  return QRKIT_OK;
}

qrkit_status composed_solve_r(qrkit_ctx* ctx, const void* qtb, void* p) {
  if (ctx->precision == QRKIT_FP64) return solve_r_typed<double>(ctx, qtb, p);
  return solve_r_typed<float>(ctx, qtb, p);
}

// Distributed pieces (a dense S whose rows are split over several contexts): the squared column
// sums of J, the R of the reduced shared block, and the block unknowns for given shared ones.
qrkit_status composed_column_sumsq(qrkit_ctx* ctx, const void* J, const void* S, double* out) {
  Composed& C = ctx->comp;
  const int64_t N = ctx->plan.cols + ctx->plan.s.shared_cols;
  qrkit_status rc;
  if ((rc = ensure(ctx, C.D, (size_t)N * sizeof(double), "D")) != QRKIT_OK) return rc;
  if ((rc = composed_column_norms(ctx, J, S, (double*)C.D.ptr)) != QRKIT_OK) return rc;
  QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(out, C.sq.ptr, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice,
                                      ctx->stream));
  return QRKIT_OK;
}

template <typename T>
__global__ void norms_from_sumsq_kernel(const double* sq, T* D, int64_t n) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double d = sqrt(sq[j]);
  D[j] = (T)(d == 0.0 ? 1.0 : d);   // zero column norm -> 1
}

qrkit_status composed_norms_from_sumsq(qrkit_ctx* ctx, const double* sq, int64_t n, void* D) {
  if (ctx->precision == QRKIT_FP64)
    LAUNCH(ctx, norms_from_sumsq_kernel<double><<<blocks_for(n, 256), 256, 0, ctx->stream>>>(sq, (double*)D, n));
  else
    LAUNCH(ctx, norms_from_sumsq_kernel<float><<<blocks_for(n, 256), 256, 0, ctx->stream>>>(sq, (float*)D, n));
  return QRKIT_OK;
}

template <typename T>
__global__ void copy_upper_kernel(const T* X, int64_t ld, int s, T* R) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)s * s) return;
  const int i = (int)(e % s), j = (int)(e / s);
  R[e] = i <= j ? X[(int64_t)j * ld + i] : T(0);
}

qrkit_status composed_reduced_r(qrkit_ctx* ctx, void* R) {
  Composed& C = ctx->comp;
  const int s = (int)ctx->plan.s.shared_cols;
  const TsqrLevel& top = C.levels.back();
  const void* src = C.panels.empty() ? top.X.ptr : C.Rs.ptr;
  const int64_t ld = C.panels.empty() ? top.ld : s;
  if (ctx->precision == QRKIT_FP64)
    LAUNCH(ctx, copy_upper_kernel<double><<<blocks_for((int64_t)s * s, 256), 256, 0, ctx->stream>>>(
                    (const double*)src, ld, s, (double*)R));
  else
    LAUNCH(ctx, copy_upper_kernel<float><<<blocks_for((int64_t)s * s, 256), 256, 0, ctx->stream>>>(
                    (const float*)src, ld, s, (float*)R));
  return QRKIT_OK;
}

template <typename T>
static qrkit_status solve_blocks_typed(qrkit_ctx* ctx, const void* qtb, void* p) {
  Plan& P = ctx->plan;
  ComposedView<T> V = view<T>(ctx, nullptr, nullptr);
  FactorOut<T> O = fout<T>(ctx);
  T* x = (T*)p;
  LAUNCH(ctx, block_backsub_kernel<T><<<blocks_for(P.K, 64), 64, 0, ctx->stream>>>(
                  V, O, (const T*)qtb, V.s ? x + P.cols : nullptr, x, 0));
  return QRKIT_OK;
}

qrkit_status composed_solve_blocks(qrkit_ctx* ctx, const void* qtb, void* p) {
  if (ctx->precision == QRKIT_FP64) return solve_blocks_typed<double>(ctx, qtb, p);
  return solve_blocks_typed<float>(ctx, qtb, p);
}

}  // namespace qrkit
