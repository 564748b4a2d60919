// Column-panel TSQR of the dense reduced shared block (float, s a multiple of 32, 256-row tiles).
// The reduced block is factored by panels of 32 columns (Sec. 2, compact WY): each panel is a
// TSQR whose tiles are factored by tsqr_panel_tile_kernel (Householder QR with the columns in
// registers, then the panel's T), and after every TSQR level tsqr_panel_apply_kernel applies the
// tiles' Q^T = I - Y T^T Y^T to the later columns:
//   1. W = Y^T C for the trailing columns C, then Z = T^T W (CUDA cores);
//   2. C -= Y Z on the tensor cores: tcgen05.mma kind::tf32 with the 3xTF32 split
//      (Y = Y_hi + Y_lo, Z = Z_hi + Z_lo, Y Z ~ Y_hi Z_hi + Y_hi Z_lo + Y_lo Z_hi), FP32
//      accumulation in TMEM, M = 128 rows per half tile, K = 32, N = trailing columns; the
//      product is read back with tcgen05.ld and subtracted in shared memory.
// Operands are staged in shared memory in the canonical K-major no-swizzle layout (8-row x
// 16-byte core matrices) and described by tcgen05 shared-memory descriptors.  Tiles arrive by
// bulk copies (TMA).  The outputs are those of any Householder TSQR (V below / R on and above
// the diagonal, tau per column, the tile's R rows to the next TSQR level), so Q^T b and the
// solves apply it reflector by reflector.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "device_util.cuh"
#include "internal.h"

namespace qrkit {
namespace {

constexpr int kRows = 256;      // tile rows (two MMA halves of 128)
constexpr int kNb = 32;         // panel width = MMA K
constexpr int kThr = 512;       // threads of the panel update (16 warps)
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of (row, k) in a K-major, no-swizzle operand with K = 32: 8-row x 16-byte core
// matrices, adjacent in K at 128 B (LBO), 8-row groups at 1024 B (SBO).
__device__ __forceinline__ uint32_t koff(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;    // leading byte offset: next core matrix in K
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version
  return d;                           // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
  // D f32 (bits 4-5 = 1), A and B tf32 (= 2 at bits 7-9, 10-12), both K-major, N >> 3 at
  // bits 17-22, M >> 4 at bits 24-28
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Sum over the warp of 32 values per lane, transposed: lane l ends with the sum over all lanes
// of v[l] (31 shuffles: at each halving a lane keeps the half of the pairs its bit selects).
__device__ __forceinline__ float transpose_reduce(float (&v)[32], int lane) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const bool upper = (lane & d) != 0;
#pragma unroll
    for (int k = 0; k < d; ++k) {
      const float send = upper ? v[k] : v[k + d];
      const float keep = upper ? v[k + d] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, d);
    }
  }
  return v[0];
}

__device__ __forceinline__ void tc_record(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Rows [r0, r0 + r) of `cols` columns of a column-major matrix (ld a multiple of 4, 16-byte
// aligned base) into shared memory at a column stride of kRows, by bulk copies (TMA) on one
// mbarrier; issued by one thread.  Each copy takes the rows rounded up to a multiple of 4 (inside
// the padded column), so the caller zeroes rows r .. kRows - 1 after the wait.
__device__ __forceinline__ uint32_t column_bytes(int r) { return (uint32_t)((r + 3) & ~3) * 4u; }
__device__ __forceinline__ void stage_columns(float* dst, const float* src, int64_t ld, int64_t r0, int r,
                                              int cols, uint64_t* bar) {
  const uint32_t cb = column_bytes(r);
  for (int c = 0; c < cols; ++c) dev::bulk_g2s(dst + (size_t)c * kRows, src + (int64_t)c * ld + r0, cb, bar);
}

// Bounded wait for the mbarrier's phase `parity`; false if the limit ran out.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (dev::mbar_try_wait(bar, parity)) return true;
  return false;
}

// ---- Column-panel TSQR: the QR of one 256-row tile of a 32-column panel ----
//
// Householder QR (Sec. 2) of a 256 x 32 tile with its columns in registers: column j lives on
// warp j % 16, row i = lane + 32 u (u < 8) of it on the lane.  At step k the reflector v_k of
// column k goes through shared memory (two alternating slots); every warp applies it to its
// columns after k (a dot product, then an axpy, in registers) and takes the products
// G[c][k] = v_c^T v_k of its columns c before k, its two reductions interleaved; the warp that
// holds column k + 1 forms the next reflector right after updating it.  Then the compact-WY T
// (T[k][k] = tau_k, column k of the strict upper part = -tau_k T[:, :k] G[:k, k]) for the panel
// update.  Outputs as any TSQR tile: reflectors below / R on and above the diagonal in place,
// tau per column, T, the R rows to the next level.
constexpr int kPT = 512;        // threads of a panel tile (16 warps, two columns each)
constexpr int kPad = kNb + 1;   // row stride of G and T in shared memory (conflict-free rows)

size_t panel_tile_smem() {
  return (size_t)kRows * kNb * 4 + 2 * (size_t)kRows * 4 + 2 * (size_t)kNb * kPad * 4;
}

__global__ void __launch_bounds__(kPT, 1)
tsqr_panel_tile_kernel(float* X, int64_t ld, int64_t M, float* taus, float* Xn, int64_t ldn, float* Tout,
                       int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* A = reinterpret_cast<float*>(smem_raw);   // 256 x 32, column-major
  float* V = A + kRows * kNb;                      // two reflector slots of 256
  float* Gs = V + 2 * kRows;                       // 32 x 33: G[m][k] at m * kPad + k
  float* Tm = Gs + kNb * kPad;                     // 32 x 33: T[l][k] at l * kPad + k
  __shared__ float tslot[2];
  __shared__ float tau_s[kNb];
  __shared__ __align__(8) uint64_t mbar_ld;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  const int r = (int)(M - r0 < (int64_t)kRows ? M - r0 : (int64_t)kRows);
  const int kmax = r < kNb ? r : kNb;
  const bool bulk = (ld & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar_ld)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (bulk) {
      dev::mbar_expect_tx(&mbar_ld, column_bytes(r) * (uint32_t)kNb);
      stage_columns(A, X, ld, r0, r, kNb, &mbar_ld);
    }
  }
  if (!bulk)
    for (int e = tid; e < kRows * kNb; e += kPT) {
      const int c = e / kRows, i = e % kRows;
      A[e] = i < r ? X[(int64_t)c * ld + r0 + i] : 0.f;
    }
  __syncthreads();
  if (bulk) {
    const bool ok = wait_phase(&mbar_ld, 0u);
    if (__syncthreads_or(!ok)) {
      // the copies may still be in flight: one more bounded wait before the CTA exits
      if (tid == 0) tc_record(status, QRKIT_ETIMEOUT);
      wait_phase(&mbar_ld, 0u);
      return;
    }
    for (int e = tid; e < (kRows - r) * kNb; e += kPT) {   // rows past the tile's end
      const int c = e / (kRows - r), i = r + e % (kRows - r);
      A[c * kRows + i] = 0.f;
    }
    __syncthreads();
  }
  // the warp's two columns in registers
  float a0[kRows / 32], a1[kRows / 32];
#pragma unroll
  for (int u = 0; u < kRows / 32; ++u) {
    a0[u] = A[warp * kRows + lane + 32 * u];
    a1[u] = A[(warp + 16) * kRows + lane + 32 * u];
  }
  // the reflector of column k from its register column a (its owner warp): the column below k
  // scaled to v (v_k = 1, stored implicitly), beta on the diagonal, v written to slot `slot`
  auto form = [&](int k, float (&a)[kRows / 32], int slot) {
    float sq = 0.f, ak = 0.f;
#pragma unroll
    for (int u = 0; u < kRows / 32; ++u) {
      const int i = lane + 32 * u;
      if (i > k) sq += a[u] * a[u];
      if (u == (k >> 5)) ak = a[u];
    }
    sq = warp_sum(sq);
    const float alpha = __shfl_sync(0xffffffffu, ak, k & 31);
    const float norm = sqrtf(alpha * alpha + sq);
    float beta = 0.f, t = 0.f, scale = 0.f;
    if (norm != 0.f) {
      beta = alpha >= 0.f ? -norm : norm;
      t = (beta - alpha) / beta;
      scale = 1.f / (alpha - beta);
    }
#pragma unroll
    for (int u = 0; u < kRows / 32; ++u) {
      const int i = lane + 32 * u;
      if (i > k) a[u] *= scale;
      else if (i == k) a[u] = beta;
      V[slot * kRows + i] = i > k ? a[u] : (i == k ? 1.f : 0.f);
    }
    if (lane == 0) {
      tslot[slot] = t;
      tau_s[k] = t;
      taus[(int64_t)blockIdx.x * kNb + k] = t;
    }
  };
  for (int e = tid; e < kNb * kPad; e += kPT) Gs[e] = 0.f;
  if (warp == 0 && kmax > 0) form(0, a0, 0);
  const int c0 = warp, c1 = warp + 16;   // the warp's columns (a0, a1)
  for (int k = 0; k < kmax; ++k) {
    __syncthreads();   // reflector k in slot k & 1; column k + 1 not yet updated
    const int slot = k & 1;
    const float t = tslot[slot];
    // v_k against each own column: the column itself if it is after k (to update it: a -= t
    // (v^T a) v), its reflector y_c (1 at row c, v_c below, 0 above) if it is before k (G[c][k])
    float v[kRows / 32], p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int u = 0; u < kRows / 32; ++u) {
      const int i = lane + 32 * u;
      v[u] = V[slot * kRows + i];
      const float y0 = c0 > k ? a0[u] : (i > c0 ? a0[u] : (i == c0 ? 1.f : 0.f));
      const float y1 = c1 > k ? a1[u] : (i > c1 ? a1[u] : (i == c1 ? 1.f : 0.f));
      p0 += v[u] * y0;
      p1 += v[u] * y1;
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      p0 += __shfl_xor_sync(0xffffffffu, p0, d);
      p1 += __shfl_xor_sync(0xffffffffu, p1, d);
    }
    if (c0 > k) {
      const float w = p0 * t;
#pragma unroll
      for (int u = 0; u < kRows / 32; ++u) a0[u] -= w * v[u];
    } else if (c0 < k && lane == 0) {
      Gs[c0 * kPad + k] = p0;
    }
    if (c1 > k) {
      const float w = p1 * t;
#pragma unroll
      for (int u = 0; u < kRows / 32; ++u) a1[u] -= w * v[u];
    } else if (c1 < k && lane == 0) {
      Gs[c1 * kPad + k] = p1;
    }
    if (k + 1 < kmax && ((k + 1) & 15) == warp) {
      if (k + 1 < 16) form(k + 1, a0, slot ^ 1);
      else form(k + 1, a1, slot ^ 1);
    }
  }
#pragma unroll
  for (int u = 0; u < kRows / 32; ++u) {
    A[warp * kRows + lane + 32 * u] = a0[u];
    A[(warp + 16) * kRows + lane + 32 * u] = a1[u];
  }
  for (int e = tid; e < kNb * kPad; e += kPT) Tm[e] = 0.f;
  __syncthreads();
  // T, column by column on warp 0 (lane l holds row l).  The sum runs over all 32 m: T[l][m]
  // is still zero for m >= k and below the diagonal, and G[m][k] for m >= k.
  if (warp == 0) {
    for (int k = 0; k < kNb; ++k) {
      const float tk = k < kmax ? tau_s[k] : 0.f;
      float q[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int m = 0; m < kNb; ++m) q[m & 3] += Tm[lane * kPad + m] * Gs[m * kPad + k];
      const float v = -((q[0] + q[1]) + (q[2] + q[3])) * tk;
      __syncwarp();
      if (lane < k) Tm[lane * kPad + k] = v;
      if (lane == k) Tm[k * kPad + k] = tk;
      __syncwarp();
    }
  }
  __syncthreads();
  if (Tout)
    for (int e = tid; e < kNb * kNb; e += kPT)
      Tout[(int64_t)blockIdx.x * (kNb * kNb) + e] = Tm[(e / kNb) * kPad + e % kNb];
  for (int e = tid; e < r * kNb; e += kPT) {
    const int c = e / r, i = e % r;
    X[(int64_t)c * ld + r0 + i] = A[c * kRows + i];
  }
  if (Xn) {
    const int64_t n0 = (int64_t)blockIdx.x * kNb;
    for (int e = tid; e < kmax * kNb; e += kPT) {
      const int c = e / kmax, i = e % kmax;
      Xn[(int64_t)c * ldn + n0 + i] = (c >= i) ? A[c * kRows + i] : 0.f;
    }
  }
}

// ---- Column-panel TSQR: a factored panel's tile reflectors applied to the columns after it ----
//
// One CTA takes one 256-row tile of a TSQR level and kCw of the trailing columns C (staged by
// bulk copies).  For each group of 32 reflectors of the tile's panel (Y, with the panel tile's
// T), Q_group^T C = C - Y (T^T (Y^T C)): W = Y^T C and Z = T^T W on the CUDA cores, C -= Y Z on
// the tensor cores (kind::tf32, 3xTF32, FP32 accumulation in TMEM).  The
// transformed tile's top rows (R rows of the panel) go up to the next level, the others down to
// the next panel.  Y arrives column by column in the space of its low operand half and is kept
// row-major (rows padded to kYr floats), so that a lane reads four reflectors of its row in one
// 16-byte load.
constexpr int kCw = 64;   // trailing columns per CTA
constexpr int kYr = 36;   // row stride of the row-major Y: 16-byte rows, conflict-free quarter warps

size_t panel_apply_smem() {
  return (size_t)kRows * kCw * 4 + (size_t)kRows * kYr * 4 + 2 * (size_t)kRows * kNb * 4 +
         2 * (size_t)kCw * kNb * 4 + (size_t)kNb * kNb * 4 + (size_t)kNb * kCw * 4;
}

__global__ void __launch_bounds__(kThr, 1)
tsqr_panel_apply_kernel(const float* X, int64_t ld, int64_t M, int pw, const float* Tin, int n, float* up,
                        int64_t ldu, float* down, int64_t ldd, int64_t down0, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* Cs = reinterpret_cast<float*>(smem_raw);                          // 256 x kCw, column-major
  float* Yr = Cs + kRows * kCw;                                            // 256 x 32, row-major (kYr)
  unsigned char* Yhi = reinterpret_cast<unsigned char*>(Yr + kRows * kYr);  // 256 x 32 operand
  unsigned char* Ylo = Yhi + kRows * kNb * 4;
  float* Yf = reinterpret_cast<float*>(Ylo);   // Y as copied (256 x 32, column-major), until Yr is formed
  unsigned char* Zhi = Ylo + kRows * kNb * 4;                              // kCw x 32 operand
  unsigned char* Zlo = Zhi + kCw * kNb * 4;
  float* Tm = reinterpret_cast<float*>(Zlo + kCw * kNb * 4);               // 32 x 32 (row l, col k)
  float* W = Tm + kNb * kNb;                                               // 32 x kCw, row-major
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t mbar_ld, mbar_mma;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t tile = blockIdx.x;
  const int64_t r0 = tile * kRows;
  const int r = (int)(M - r0 < (int64_t)kRows ? M - r0 : (int64_t)kRows);
  const int kmax = r < pw ? r : pw;
  const int j0 = blockIdx.y * kCw;
  const int nc = n - j0 < kCw ? n - j0 : kCw;   // a multiple of 32
  const float* Cg = X + (int64_t)(pw + j0) * ld;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(2 * kCw));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar_ld)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar_mma)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  uint32_t ph_ld = 0, ph_mma = 0;
  int pending = 0;   // 1: a bulk load, 2: the MMAs still outstanding after a timeout

  for (int p0 = 0; p0 < kmax; p0 += kNb) {
    const int nk = kmax - p0 < kNb ? kmax - p0 : kNb;
    // (a) Y of this group of reflectors (and, the first time, the tile's trailing columns)
    dev::fence_proxy_async();
    __syncthreads();   // every earlier read of Yf and Cs is done
    if (tid == 0) {
      dev::mbar_expect_tx(&mbar_ld, column_bytes(r) * (uint32_t)(nk + (p0 == 0 ? nc : 0)));
      stage_columns(Yf, X + (int64_t)p0 * ld, ld, r0, r, nk, &mbar_ld);
      if (p0 == 0) stage_columns(Cs, Cg, ld, r0, r, nc, &mbar_ld);
    }
    for (int e = tid; e < kNb * kNb; e += kThr) Tm[e] = Tin[(tile * (pw / kNb) + p0 / kNb) * (kNb * kNb) + e];
    const bool ok = wait_phase(&mbar_ld, ph_ld);
    ph_ld ^= 1u;
    if (__syncthreads_or(!ok)) {
      pending = 1;
      break;
    }
    // Y[i][l]: 1 at i = p0 + l, the stored v below, 0 above, past the tile and for l >= nk
    for (int e = tid; e < kRows * kNb; e += kThr) {
      const int l = e / kRows, i = e % kRows, d = p0 + l;
      Yr[i * kYr + l] = (l >= nk || i < d || i >= r) ? 0.f : (i == d ? 1.f : Yf[e]);
    }
    if (p0 == 0)
      for (int e = tid; e < (kRows - r) * nc; e += kThr) {
        const int c = e / (kRows - r), i = r + e % (kRows - r);
        Cs[c * kRows + i] = 0.f;
      }
    __syncthreads();
    // (b) W = Y^T C (32 x nc): a warp per pair of columns, lanes over rows p0.., each row's 32
    // reflector values in eight 16-byte loads; the 32 sums of a column reduced together
    for (int j = 2 * warp; j < nc; j += 2 * (kThr / 32)) {
      float acc0[32], acc1[32];
#pragma unroll
      for (int l = 0; l < 32; ++l) acc0[l] = acc1[l] = 0.f;
      const float* x0 = Cs + j * kRows;
      const float* x1 = x0 + kRows;
      for (int i = p0 + lane; i < kRows; i += 32) {
        const float c0 = x0[i], c1 = x1[i];
        const float4* yrow = reinterpret_cast<const float4*>(Yr + i * kYr);
#pragma unroll
        for (int q = 0; q < kNb / 4; ++q) {
          const float4 y = yrow[q];
          acc0[4 * q] += y.x * c0;
          acc0[4 * q + 1] += y.y * c0;
          acc0[4 * q + 2] += y.z * c0;
          acc0[4 * q + 3] += y.w * c0;
          acc1[4 * q] += y.x * c1;
          acc1[4 * q + 1] += y.y * c1;
          acc1[4 * q + 2] += y.z * c1;
          acc1[4 * q + 3] += y.w * c1;
        }
      }
      W[lane * kCw + j] = transpose_reduce(acc0, lane);
      W[lane * kCw + j + 1] = transpose_reduce(acc1, lane);
    }
    __syncthreads();
    // (c) Z = T^T W in place (row i of Z from rows l <= i of W)
    for (int j = tid; j < nc; j += kThr)
      for (int i = kNb - 1; i >= 0; --i) {
        float z = 0.f;
        for (int l = 0; l <= i; ++l) z += Tm[l * kNb + i] * W[l * kCw + j];
        W[i * kCw + j] = z;
      }
    __syncthreads();
    // (d) operands: Z (nc x 32, K-major) and Y (256 x 32), each split into TF32 hi + lo
    for (int e = tid; e < kNb * nc; e += kThr) {
      const int i = e / nc, j = e % nc;
      const float v = W[i * kCw + j], h = to_tf32(v);
      *reinterpret_cast<float*>(Zhi + koff(j, i)) = h;
      *reinterpret_cast<float*>(Zlo + koff(j, i)) = to_tf32(v - h);
    }
    for (int e = tid; e < kRows * kNb; e += kThr) {
      const int l = e / kRows, i = e % kRows;
      const float v = Yr[i * kYr + l], h = to_tf32(v);
      const uint32_t o = (uint32_t)(i >> 7) * (128 * kNb * 4) + koff(i & 127, l);
      *reinterpret_cast<float*>(Yhi + o) = h;
      *reinterpret_cast<float*>(Ylo + o) = to_tf32(v - h);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // (e) D_h = Y_h Z for the two 128-row halves (3 products each: hi hi, hi lo, lo hi)
    if (tid == 0) {
      const uint32_t id = idesc_tf32(128, nc);
      for (int h = 0; h < 2; ++h) {
        const uint32_t yo = (uint32_t)h * (128 * kNb * 4);
        int first = 1;
        for (int ks = 0; ks < kNb / 8; ++ks) {
          const uint32_t ko = (uint32_t)ks * 256;
          for (int sp = 0; sp < 3; ++sp) {
            const unsigned char* ya = sp == 2 ? Ylo : Yhi;
            const unsigned char* zb = sp == 1 ? Zlo : Zhi;
            const uint64_t ad = smem_desc(su32(ya) + yo + ko), bd = smem_desc(su32(zb) + ko);
            const uint32_t acc = first ? 0u : 1u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)(h * kCw)),
                "l"(ad), "l"(bd), "r"(id), "r"(acc));
            first = 0;
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(&mbar_mma)));
    }
    const bool mma_ok = wait_phase(&mbar_mma, ph_mma);
    ph_mma ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (__syncthreads_or(!mma_ok)) {
      pending = 2;
      break;
    }
    // (f) C -= D: warp w reads TMEM lanes 32 (w % 4) .. of half (w / 4) % 2, 8-column groups
    // (w / 8), (w / 8) + 2, ...
    {
      const int qd = warp & 3, h = (warp >> 2) & 1, part = warp >> 3;
      const int row = h * 128 + qd * 32 + lane;
      for (int c0 = part * 8; c0 < nc; c0 += 8 * (kThr / 256)) {
        uint32_t v[8];
        const uint32_t ta = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(h * kCw + c0);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7])
                     : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < 8; ++j) Cs[(c0 + j) * kRows + row] -= __uint_as_float(v[j]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  if (pending) {
    if (tid == 0) tc_record(status, QRKIT_ETIMEOUT);
    // what timed out may still be running: wait once more (bounded) before TMEM and shared
    // memory are given up
    if (pending == 1) wait_phase(&mbar_ld, ph_ld ^ 1u);
    else wait_phase(&mbar_mma, ph_mma ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kCw));
  if (pending) return;
  // the tile's top kmax rows up (the next level, or R_S), the others down (the next panel)
  for (int e = tid; e < r * nc; e += kThr) {
    const int c = e / r, i = e % r;
    const float v = Cs[c * kRows + i];
    if (i < kmax) up[(int64_t)(j0 + c) * ldu + tile * pw + i] = v;
    else down[(int64_t)(j0 + c) * ldd + down0 + tile * (kRows - pw) + (i - kmax)] = v;
  }
}

}  // namespace

qrkit_status tsqr_panel_apply(qrkit_ctx* ctx, const float* X, int64_t ld, int64_t M, int pw, const float* T,
                              int n, float* up, int64_t ldu, float* down, int64_t ldd, int64_t down0,
                              int64_t tiles) {
  if (n <= 0 || tiles <= 0) return QRKIT_OK;
  if ((ld & 3) != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0 || pw % kNb != 0 || n % kNb != 0 ||
      pw > kRows / 2)
    return fail(ctx, QRKIT_EINVAL, "column-panel TSQR: unaligned level matrix or panel shape");
  const size_t smem = panel_apply_smem();
  if (smem > ctx->max_smem_optin)
    return fail(ctx, QRKIT_EUNSUPPORTED, "not enough shared memory for the column-panel TSQR kernel");
  if (ctx->smem_attr[15] < smem) {
    QRKIT_CUDA_TRY(ctx, cudaFuncSetAttribute(tsqr_panel_apply_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ctx->smem_attr[15] = smem;
  }
  const dim3 grid((unsigned)tiles, (unsigned)((n + kCw - 1) / kCw));
  tsqr_panel_apply_kernel<<<grid, kThr, smem, ctx->stream>>>(X, ld, M, pw, T, n, up, ldu, down, ldd, down0,
                                                             ctx->d_status);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

qrkit_status tsqr_panel_tile(qrkit_ctx* ctx, float* X, int64_t ld, int64_t M, float* taus, float* Xn, int64_t ldn,
                             int64_t tiles, float* Tout) {
  const size_t smem = panel_tile_smem();
  if (smem > ctx->max_smem_optin)
    return fail(ctx, QRKIT_EUNSUPPORTED, "not enough shared memory for the panel tile kernel");
  if (ctx->smem_attr[13] < smem) {
    QRKIT_CUDA_TRY(ctx, cudaFuncSetAttribute(tsqr_panel_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
    ctx->smem_attr[13] = smem;
  }
  tsqr_panel_tile_kernel<<<(unsigned)tiles, kPT, smem, ctx->stream>>>(X, ld, M, taus, Xn, ldn, Tout, ctx->d_status);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

}  // namespace qrkit
