// Parallel QR of banded matrices (Sec. 4.4) by row compression and block cyclic reduction.
//
// An instance has N columns, cut into G = ceil(N / 8) blocks of 8 (the last block padded
// with "virtual" columns that carry a unit damping row and nothing else, so that the padded
// matrix has full rank and the real columns' solution is unchanged).  Every row has at most
// 8 consecutive entries, so a row whose first column lies in block g touches blocks g and
// g + 1 only.
//
//   1. compress   per block g, the Householder QR (Sec. 2) of all rows starting in block g
//                 plus the damping rows lambda^(1/2) D_j of the block's columns (the row
//                 interleave of Sec. 4.5 / 5.2) reduces them to a 16 x 16 upper-trapezoidal
//                 block row E_g = [A_g | B_g] on blocks (g, g + 1).  Large groups are split
//                 over several warps whose partial triangles are merged.
//   2. reduce     level l works on the block rows F_i of blocks b_i = i 2^l: for every odd
//                 i, QR of [F_{i-1}; F_i] with block b_i's columns first gives the 8 rows of R
//                 for b_i (coupled to b_{i-1} and b_{i+1}) and a new 16-row block row on
//                 (b_{i-1}, b_{i+1}); an unpaired last block row moves up unchanged; at one
//                 block row the last R rows come out.  All eliminations of a level run in
//                 parallel, ceil(log2 G) + 1 levels.
//   3. solve      back-substitution level by level from the top: R_bb x_b = c_b - R_left
//                 x_{b - 2^l} - R_right x_{b + 2^l} for all blocks of a level in parallel.
// The product is a QR factorization of the matrix with its columns in nested-dissection
// order (the blocks of the lowest level first), so R differs from the natural-order banded
// R; R^T R = A^T A and the solution are the same.  Every Householder vector is as long as a
// 32-row front.  Refinement solves R^T h = g level by level upwards, then R dx = h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace qrkit {
namespace {

constexpr int kCB = 8;             // columns per block
constexpr int kEW = 2 * kCB + 1;   // block row stride: A (8) | B (8) | rhs
constexpr int kRW = 3 * kCB + 1;   // R block row stride: own (8) | left (8) | right (8) | rhs

__device__ __forceinline__ void cr_record(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Square root and reciprocal of the front QR: the hardware approximations for float
// (sqrt.approx / rcp.approx, about one ulp: far below the rounding the factorization itself
// accumulates), IEEE for double.
__device__ __forceinline__ float qr_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double qr_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float qr_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double qr_rcp(double x) { return 1.0 / x; }

__host__ __device__ constexpr int pow2_ceil(int m) { return m <= 1 ? 1 : 2 * pow2_ceil((m + 1) / 2); }
__host__ __device__ constexpr int log2_exact(int p) { return p <= 1 ? 0 : 1 + log2_exact(p / 2); }

// Sums of M per-lane values over the warp, returned in every lane (v[j] = sum over lanes).
// Transpose reduction: with the values padded to P = 2^ceil(log2 M), each butterfly stage
// sends half of the remaining values to the partner lane and keeps the other half, so after
// log2 P stages each lane holds one partial sum (of value lane >> (5 - log2 P)); plain
// butterfly stages finish the sums, and one broadcast per value returns them.  About
// P - 1 + M shuffles instead of 5 M; every lane reads the same lane's sum, so all lanes hold
// the same bits.
template <typename T, int M>
__device__ __forceinline__ void warp_allreduce_many(T (&v)[M], int lane) {
  constexpr int P = pow2_ceil(M);
  constexpr int S = 5 - log2_exact(P);
  static_assert(P <= 32, "at most 32 values");
  T w[P];
#pragma unroll
  for (int i = 0; i < P; ++i) w[i] = i < M ? v[i] : T(0);
  int d = 16;
#pragma unroll
  for (int h = P / 2; h >= 1; h /= 2, d >>= 1) {
    const bool up = (lane & d) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? w[i] : w[h + i];
      const T keep = up ? w[h + i] : w[i];
      w[i] = keep + __shfl_xor_sync(0xffffffffu, send, d);
    }
  }
#pragma unroll
  for (int e = 0; e < S; ++e) {
    w[0] += __shfl_xor_sync(0xffffffffu, w[0], d);
    d >>= 1;
  }
#pragma unroll
  for (int jj = 0; jj < M; ++jj) v[jj] = __shfl_sync(0xffffffffu, w[0], jj << S);
}

// Householder QR of a 32-row front held one row per lane (a[0..NC-1] columns, a[NC] the
// right-hand side), reducing columns 0..NK-1 in order.  Row k of the result holds R's row k
// (lane k); rows below NK are zero in the reduced columns.  Column K of the recursion: its
// reflector, then the update of the NC - K trailing columns (and rhs), whose dot products
// with v are summed over the warp together.
template <typename T, int NC, int K, int NK>
__device__ __forceinline__ void warp_qr_col(T (&a)[NC + 1], int lane) {
  const T x = a[K];
  const T sq = wsum(lane > K ? x * x : T(0));
  const T alpha = __shfl_sync(0xffffffffu, x, K);
  const T norm = qr_sqrt(alpha * alpha + sq);
  T beta = T(0), tau = T(0), scale = T(0);
  if (norm != T(0)) {
    beta = alpha >= T(0) ? -norm : norm;
    tau = (beta - alpha) * qr_rcp(beta);
    scale = qr_rcp(alpha - beta);
  }
  const T v = lane > K ? x * scale : (lane == K ? T(1) : T(0));
  T dv[NC - K];
#pragma unroll
  for (int jj = 0; jj < NC - K; ++jj) dv[jj] = v * a[K + 1 + jj];
  warp_allreduce_many<T, NC - K>(dv, lane);
#pragma unroll
  for (int jj = 0; jj < NC - K; ++jj) a[K + 1 + jj] -= (dv[jj] * tau) * v;
  if (lane == K) a[K] = beta;
  else if (lane > K) a[K] = T(0);
  if constexpr (K + 1 < NK) warp_qr_col<T, NC, K + 1, NK>(a, lane);
}

template <typename T, int NC, int NK>
__device__ __forceinline__ void warp_qr(T (&a)[NC + 1], int lane) {
  warp_qr_col<T, NC, 0, NK>(a, lane);
}

template <typename T>
struct CRArgs {
  // instances
  int64_t num_inst;
  const int64_t* cols;    // N
  const int64_t* col0;    // first global column
  const int64_t* row0;    // first global row
  const int64_t* rows;    // rows of the instance
  const int64_t* blk0;    // num_inst + 1: first global block of each instance
  int64_t total_blocks;
  // rows: explicit starts (global columns, sorted per instance) or implicit floor(i / rpc)
  const int64_t* starts;
  int rpc;
  int w;
  const T* J;             // rows x w
  const T* b;             // rows
  const double* D;        // global columns (damping rows when lam > 0)
  double lam;
  int splits;             // warps per block in the compression
  // work space
  int64_t* grp_lo;        // total_blocks: first row of each block's group (explicit starts)
  T* P;                   // total_blocks x splits x 16 x kEW partial triangles
  T* F0;                  // total_blocks x 16 x kEW block rows (two buffers)
  T* F1;
  T* Rb;                  // total_blocks x 8 x kRW
  T* xp;                  // total_blocks x 8 padded solution / rhs work
  T* hp;                  // total_blocks x 8
  double* res2;           // per instance
  int* status;
};

__device__ __forceinline__ int64_t inst_of_block(const int64_t* blk0, int64_t ninst, int64_t gb) {
  int64_t lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (blk0[mid] <= gb) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// First row of each block's group: lower bound of 8 g among the instance's sorted starts.
template <typename T>
__global__ void cr_ranges_kernel(CRArgs<T> A) {
  const int64_t gb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gb >= A.total_blocks) return;
  const int64_t k = inst_of_block(A.blk0, A.num_inst, gb);
  const int64_t g = gb - A.blk0[k];
  const int64_t key = A.col0[k] + (int64_t)kCB * g;
  int64_t lo = A.row0[k], hi = A.row0[k] + A.rows[k];
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (A.starts[mid] < key) lo = mid + 1; else hi = mid;
  }
  A.grp_lo[gb] = lo;
}

template <typename T>
__device__ __forceinline__ void group_rows(const CRArgs<T>& A, int64_t k, int64_t g, int64_t gb, int64_t& lo,
                                           int64_t& hi) {
  const int64_t nb = A.blk0[k + 1] - A.blk0[k];
  const int64_t end = A.row0[k] + A.rows[k];
  if (A.starts) {
    lo = A.grp_lo[gb];
    hi = g + 1 < nb ? A.grp_lo[gb + 1] : end;
  } else {
    const int64_t r0 = A.row0[k] + (int64_t)A.rpc * kCB * g;
    lo = r0 < end ? r0 : end;
    const int64_t r1 = r0 + (int64_t)A.rpc * kCB;
    hi = r1 < end ? r1 : end;
  }
}

// ---- 1. compression of blocks with few rows: one thread per block, rows merged one at a time into an
// upper-triangular 16 x 16 (+ rhs) block row by 2 x 2 orthogonal rotations (the 2-element
// Householder reflections of sparse row-merge QR); the triangle lives in shared memory,
// element-major over the CTA's threads so that a warp's accesses hit distinct banks. ----
constexpr int kTriElems = 16 * 17 - 120;   // packed upper triangle incl. rhs: rows k = 0..15, cols k..16
constexpr int kCompThreads = 64;

__host__ __device__ constexpr int tri_off(int k, int j) { return k * 17 - (k * (k - 1)) / 2 + (j - k); }

template <typename T>
__device__ __forceinline__ void rot_coeffs(T alpha, T beta, T& c, T& s, T& r);
template <>
__device__ __forceinline__ void rot_coeffs<float>(float alpha, float beta, float& c, float& s, float& r) {
  const float n2 = alpha * alpha + beta * beta;
  const float rr = rsqrtf(n2);
  c = alpha * rr;
  s = beta * rr;
  r = n2 * rr;
}
template <>
__device__ __forceinline__ void rot_coeffs<double>(double alpha, double beta, double& c, double& s, double& r) {
  r = sqrt(alpha * alpha + beta * beta);
  c = alpha / r;
  s = beta / r;
}

// Merge row a (16 columns + rhs at 16, nonzero from column o on) into the triangle Tr
// (element e of this thread at Tr[e * kCompThreads]); returns the squared leftover rhs.
template <typename T>
__device__ __forceinline__ double merge_row(T* Tr, T (&a)[17], int o) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k >= o && a[k] != T(0)) {
      T c, sn, r;
      rot_coeffs<T>(Tr[tri_off(k, k) * kCompThreads], a[k], c, sn, r);
      Tr[tri_off(k, k) * kCompThreads] = r;
      a[k] = T(0);
#pragma unroll
      for (int j = k + 1; j < 17; ++j) {
        const T t = Tr[tri_off(k, j) * kCompThreads];
        Tr[tri_off(k, j) * kCompThreads] = c * t + sn * a[j];
        a[j] = c * a[j] - sn * t;
      }
    }
  }
  return (double)a[16] * (double)a[16];
}

template <typename T>
__device__ __forceinline__ void damping_rows(const CRArgs<T>& A, T* Tr, int64_t g, int64_t N, int64_t c0,
                                             double& res) {
  const bool damp = A.lam > 0.0;
  const double lam_half = sqrt(A.lam);
#pragma unroll 1
  for (int q = 0; q < kCB; ++q) {
    const int64_t col = (int64_t)kCB * g + q;
    T v = T(0);
    if (col >= N) v = T(1);   // padding column: unit row
    else if (damp) v = (T)(lam_half * A.D[c0 + col]);
    T a[17];
#pragma unroll
    for (int j = 0; j < 17; ++j) a[j] = j == q ? v : T(0);
    res += merge_row(Tr, a, q);
  }
}

template <typename T>
__device__ __forceinline__ void store_block_row(T* dst, const T* Tr) {
  // 16 rows x (16 + rhs), zeros below the diagonal
#pragma unroll
  for (int k = 0; k < 16; ++k)
#pragma unroll
    for (int j = 0; j < 17; ++j) dst[k * kEW + j] = j >= k ? Tr[tri_off(k, j) * kCompThreads] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(kCompThreads) cr_compress_kernel(CRArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Tr = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
  const int64_t item = (int64_t)blockIdx.x * kCompThreads + threadIdx.x;
  if (item >= A.total_blocks * A.splits) return;
  const int64_t gb = item / A.splits;
  const int s = (int)(item - gb * A.splits);
  const int64_t k = inst_of_block(A.blk0, A.num_inst, gb);
  const int64_t g = gb - A.blk0[k];
  const int64_t N = A.cols[k], c0 = A.col0[k];
  int64_t lo, hi;
  group_rows(A, k, g, gb, lo, hi);
  const int64_t len = hi - lo;
  const int64_t r_begin = lo + len * s / A.splits, r_end = lo + len * (s + 1) / A.splits;
#pragma unroll
  for (int e = 0; e < kTriElems; ++e) Tr[e * kCompThreads] = T(0);
  double res = 0.0;
  bool bad = false;
#pragma unroll 1
  for (int64_t r = r_begin; r < r_end; ++r) {
    const int64_t st = A.starts ? A.starts[r] - c0 : (r - A.row0[k]) / A.rpc;
    const int64_t o = st - (int64_t)kCB * g;
    if (o < 0 || o >= kCB) {
      bad = true;
      continue;
    }
    // the row over the block row's 16 columns: its w values start at column o
    T a[17];
    const T* src = A.J + r * A.w;
#pragma unroll
    for (int cc = 0; cc < 2 * kCB; ++cc) {
      const int64_t q = cc - o;
      a[cc] = (q >= 0 && q < A.w && st + q < N) ? src[q] : T(0);
    }
    a[16] = A.b[r];
    res += merge_row(Tr, a, (int)o);
  }
  if (bad) cr_record(A.status, QRKIT_EINVAL);
  if (A.splits == 1) {
    // the block's damping rows complete its block row
    damping_rows(A, Tr, g, N, c0, res);
    store_block_row(A.F0 + gb * 16 * kEW, Tr);
  } else {
    store_block_row(A.P + (gb * A.splits + s) * 16 * kEW, Tr);
  }
  if (res != 0.0) atomicAdd(A.res2 + k, res);
}

// ---- 1'. compression for row-heavy blocks: one warp per (block, split), 16 rows at a time
// reduced by the warp-level Householder QR (one row per lane); the partial triangles of the
// splits are merged by one warp per block, with the damping rows. ----
template <typename T>
__global__ void __launch_bounds__(128) cr_compress_warp_kernel(CRArgs<T> A) {
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= A.total_blocks * A.splits) return;
  const int64_t gb = item / A.splits;
  const int s = (int)(item - gb * A.splits);
  const int64_t k = inst_of_block(A.blk0, A.num_inst, gb);
  const int64_t g = gb - A.blk0[k];
  const int64_t N = A.cols[k], c0 = A.col0[k];
  int64_t lo, hi;
  group_rows(A, k, g, gb, lo, hi);
  const int64_t len = hi - lo;
  const int64_t r_begin = lo + len * s / A.splits, r_end = lo + len * (s + 1) / A.splits;
  T a[2 * kCB + 1];
#pragma unroll
  for (int q = 0; q <= 2 * kCB; ++q) a[q] = T(0);
  double res = 0.0;
  bool bad = false;
  for (int64_t base = r_begin; base < r_end; base += 16) {
    if (lane >= 16) {
      const int64_t r = base + (lane - 16);
      if (r < r_end) {
        const int64_t st = A.starts ? A.starts[r] - c0 : (r - A.row0[k]) / A.rpc;
        const int64_t o = st - (int64_t)kCB * g;
        if (o < 0 || o >= kCB) {
          bad = true;
        } else {
          const T* src = A.J + r * A.w;
#pragma unroll
          for (int q = 0; q < kCB; ++q)
            if (q < A.w && st + q < N) {
              const int c = (int)o + q;
#pragma unroll
              for (int cc = 0; cc < 2 * kCB; ++cc)
                if (cc == c) a[cc] = src[q];
            }
          a[2 * kCB] = A.b[r];
        }
      }
    }
    warp_qr<T, 2 * kCB, 2 * kCB>(a, lane);
    if (lane >= 16) {
      res += (double)a[2 * kCB] * (double)a[2 * kCB];
#pragma unroll
      for (int q = 0; q <= 2 * kCB; ++q) a[q] = T(0);
    }
  }
  if (bad) cr_record(A.status, QRKIT_EINVAL);
  if (lane < 16) {
    T* dst = A.P + ((gb * A.splits + s) * 16 + lane) * kEW;
#pragma unroll
    for (int q = 0; q <= 2 * kCB; ++q) dst[q] = a[q];
  }
  res = wsum(res);
  if (lane == 0 && res != 0.0) atomicAdd(A.res2 + k, res);
  (void)c0;
}

// 1b. one warp per block: merge the partial triangles and the damping rows into E_g.
template <typename T>
__global__ void __launch_bounds__(128) cr_merge_warp_kernel(CRArgs<T> A) {
  const int64_t gb = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gb >= A.total_blocks) return;
  const int64_t k = inst_of_block(A.blk0, A.num_inst, gb);
  const int64_t g = gb - A.blk0[k];
  const int64_t N = A.cols[k], c0 = A.col0[k];
  T a[2 * kCB + 1];
#pragma unroll
  for (int q = 0; q <= 2 * kCB; ++q) a[q] = T(0);
  if (lane < 16) {
    const T* src = A.P + ((gb * A.splits) * 16 + lane) * kEW;
#pragma unroll
    for (int q = 0; q <= 2 * kCB; ++q) a[q] = src[q];
  }
  double res = 0.0;
  const bool damp = A.lam > 0.0;
  const double lam_half = sqrt(A.lam);
  for (int s = 1; s <= A.splits; ++s) {
    if (lane >= 16) {
      if (s < A.splits) {
        const T* src = A.P + ((gb * A.splits + s) * 16 + (lane - 16)) * kEW;
#pragma unroll
        for (int q = 0; q <= 2 * kCB; ++q) a[q] = src[q];
      } else if (lane < 16 + kCB) {
        // damping rows of the block's columns; unit rows for virtual columns
        const int q0 = lane - 16;
        const int64_t col = (int64_t)kCB * g + q0;
        T v = T(0);
        if (col >= N) v = T(1);
        else if (damp) v = (T)(lam_half * A.D[c0 + col]);
#pragma unroll
        for (int q = 0; q < kCB; ++q)
          if (q == q0) a[q] = v;
      }
    }
    warp_qr<T, 2 * kCB, 2 * kCB>(a, lane);
    if (lane >= 16) {
      res += (double)a[2 * kCB] * (double)a[2 * kCB];
#pragma unroll
      for (int q = 0; q <= 2 * kCB; ++q) a[q] = T(0);
    }
  }
  if (lane < 16) {
    T* dst = A.F0 + (gb * 16 + lane) * kEW;
#pragma unroll
    for (int q = 0; q <= 2 * kCB; ++q) dst[q] = a[q];
  }
  res = wsum(res);
  if (lane == 0 && res != 0.0) atomicAdd(A.res2 + k, res);
}

// Work items of a level: inst << 32 | i << 2 | kind (0 eliminate odd i, 1 move up, 2 last).
__device__ __forceinline__ void decode(int64_t it, int64_t& k, int64_t& i, int& kind) {
  k = it >> 32;
  i = (it >> 2) & 0x3fffffff;
  kind = (int)(it & 3);
}

// 2. one warp per work item of level l.
template <typename T>
__global__ void __launch_bounds__(128) cr_level_kernel(CRArgs<T> A, const int64_t* items, int64_t nitems,
                                                       int level, const T* Fc, T* Fn) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nitems) return;
  int64_t k, i;
  int kind;
  decode(items[w], k, i, kind);
  const int64_t b0 = A.blk0[k];
  if (kind == 1) {   // unpaired last block row: moves up unchanged
    if (lane < 16) {
      const T* src = Fc + ((b0 + i) * 16 + lane) * kEW;
      T* dst = Fn + ((b0 + i / 2) * 16 + lane) * kEW;
#pragma unroll
      for (int q = 0; q < kEW; ++q) dst[q] = src[q];
    }
    return;
  }
  // front columns: own block (0..7) | left block (8..15) | right block (16..23) | rhs (24)
  T a[3 * kCB + 1];
#pragma unroll
  for (int q = 0; q <= 3 * kCB; ++q) a[q] = T(0);
  if (lane < 16) {
    if (kind == 0) {   // F_{i-1} = [A on left | B on own]
      const T* src = Fc + ((b0 + i - 1) * 16 + lane) * kEW;
#pragma unroll
      for (int q = 0; q < kCB; ++q) {
        a[kCB + q] = src[q];
        a[q] = src[kCB + q];
      }
      a[3 * kCB] = src[2 * kCB];
    }
  } else {             // F_i = [A on own | B on right]
    const T* src = Fc + ((b0 + i) * 16 + (lane - 16)) * kEW;
#pragma unroll
    for (int q = 0; q < kCB; ++q) {
      a[q] = src[q];
      a[2 * kCB + q] = src[kCB + q];
    }
    a[3 * kCB] = src[2 * kCB];
  }
  warp_qr<T, 3 * kCB, 3 * kCB>(a, lane);
  const int64_t blk = b0 + (i << level);
  if (lane < kCB) {
    T* dst = A.Rb + (blk * kCB + lane) * kRW;
#pragma unroll
    for (int q = 0; q <= 3 * kCB; ++q) dst[q] = a[q];
  }
  double res = 0.0;
  if (kind == 0) {
    if (lane >= kCB && lane < kCB + 16) {
      T* dst = Fn + ((b0 + (i - 1) / 2) * 16 + (lane - kCB)) * kEW;
#pragma unroll
      for (int q = 0; q < kCB; ++q) {
        dst[q] = a[kCB + q];
        dst[kCB + q] = a[2 * kCB + q];
      }
      dst[2 * kCB] = a[3 * kCB];
    } else if (lane >= kCB + 16) {
      res = (double)a[3 * kCB] * (double)a[3 * kCB];
    }
  } else if (lane >= kCB) {
    res = (double)a[3 * kCB] * (double)a[3 * kCB];
  }
  res = wsum(res);
  if (lane == 0 && res != 0.0) atomicAdd(A.res2 + k, res);
}

// 3. back-substitution of one level: eight threads per eliminated block, thread q owns row q
// of the block's R (own | left | right | rhs): the couplings to the neighbours' solutions
// are row-local, the triangular solve broadcasts each x_t to the block's threads (width-8
// shuffles).  rhs from the R rows' own column (c) or from hp; writes xp (padded) and, for
// real columns, x.  Threads past the last item run the shuffles with nothing to do.
constexpr int kItemThreads = kCB;

template <typename T>
__global__ void cr_backsub_kernel(CRArgs<T> A, const int64_t* items, int64_t nitems, int level, int use_hp,
                                  T* x) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t w = tid / kItemThreads;
  const int q = (int)(tid % kItemThreads);
  int64_t k = 0, i = 0;
  int kind = 1;
  if (w < nitems) decode(items[w], k, i, kind);
  const bool act = kind != 1;
  const int64_t b0 = act ? A.blk0[k] : 0, N = act ? A.cols[k] : 0;
  const int64_t G = (N + kCB - 1) / kCB;
  const int64_t beta = i << level, step = (int64_t)1 << level;
  const T* Rq = A.Rb + ((b0 + beta) * kCB + q) * kRW;
  T y = T(0), diag = T(1);
  T rq[kCB];
#pragma unroll
  for (int t = 0; t < kCB; ++t) rq[t] = T(0);
  if (act) {
    y = use_hp ? A.hp[(b0 + beta) * kCB + q] : Rq[3 * kCB];
    if (kind == 0) {
      const T* xl = A.xp + (b0 + beta - step) * kCB;
#pragma unroll
      for (int t = 0; t < kCB; ++t) y -= Rq[kCB + t] * xl[t];
    }
    if (beta + step < G) {
      const T* xr = A.xp + (b0 + beta + step) * kCB;
#pragma unroll
      for (int t = 0; t < kCB; ++t) y -= Rq[2 * kCB + t] * xr[t];
    }
#pragma unroll
    for (int t = 0; t < kCB; ++t) rq[t] = t > q ? Rq[t] : T(0);
    diag = Rq[q];
    if (diag == T(0)) cr_record(A.status, QRKIT_ESINGULAR);
  }
  T xq = T(0);
#pragma unroll
  for (int t = kCB - 1; t >= 0; --t) {   // x_t = (y_t - sum_{u > t} R_tu x_u) / R_tt, bottom up
    if (q == t) xq = y / diag;
    const T xt = __shfl_sync(0xffffffffu, xq, t, kItemThreads);
    y -= rq[t] * xt;                      // rq[t] = 0 unless t > q
  }
  if (act) {
    A.xp[(b0 + beta) * kCB + q] = xq;
    if (x && kCB * beta + q < N) x[A.col0[k] + kCB * beta + q] = xq;
  }
}

// Refinement, R^T h = g upwards: per level, h_b = R_bb^{-T} g_b for the eliminated blocks ...
// (eight threads per block; thread q solves for h_q after the h_t, t < q, are broadcast)
template <typename T>
__global__ void cr_rt_kernel(CRArgs<T> A, const int64_t* items, int64_t nitems, int level) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t w = tid / kItemThreads;
  const int q = (int)(tid % kItemThreads);
  int64_t k = 0, i = 0;
  int kind = 1;
  if (w < nitems) decode(items[w], k, i, kind);
  const bool act = kind != 1;
  const int64_t blk = act ? A.blk0[k] + (i << level) : 0;
  const T* R = A.Rb + blk * kCB * kRW;
  T v = T(0), diag = T(1);
  T col[kCB];   // column q of R above the diagonal: R_tq, t < q
#pragma unroll
  for (int t = 0; t < kCB; ++t) col[t] = T(0);
  if (act) {
    v = A.xp[blk * kCB + q];   // xp holds the updated g during the upward sweep
#pragma unroll
    for (int t = 0; t < kCB; ++t) col[t] = t < q ? R[t * kRW + q] : T(0);
    diag = R[q * kRW + q];
  }
  T hq = T(0);
#pragma unroll
  for (int t = 0; t < kCB; ++t) {   // h_t = (g_t - sum_{u < t} R_ut h_u) / R_tt, top down
    if (q == t) hq = v / diag;
    const T ht = __shfl_sync(0xffffffffu, hq, t, kItemThreads);
    v -= col[t] * ht;                // col[t] = 0 unless t < q
  }
  if (act) A.hp[blk * kCB + q] = hq;
}

// ... then the blocks that stay (even j at level l) subtract their neighbours' couplings:
// g_{b_j} -= R_{b_{j-1}}.right^T h_{b_{j-1}} + R_{b_{j+1}}.left^T h_{b_{j+1}}  (eight threads
// per block, thread q one entry of g).
template <typename T>
__global__ void cr_rt_update_kernel(CRArgs<T> A, const int64_t* items, int64_t nitems, int level) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t w = tid / kItemThreads;
  const int q = (int)(tid % kItemThreads);
  if (w >= nitems) return;
  const int64_t k = items[w] >> 32, j = items[w] & 0xffffffff;
  const int64_t b0 = A.blk0[k], N = A.cols[k];
  const int64_t G = (N + kCB - 1) / kCB;
  const int64_t Gl = (G + ((int64_t)1 << level) - 1) >> level;
  T* g = A.xp + (b0 + (j << level)) * kCB;
  T acc = g[q];
  if (j >= 1) {
    const int64_t nb = b0 + ((j - 1) << level);
    const T* R = A.Rb + nb * kCB * kRW;
    const T* h = A.hp + nb * kCB;
#pragma unroll
    for (int t = 0; t < kCB; ++t) acc -= R[t * kRW + 2 * kCB + q] * h[t];
  }
  if (j + 1 < Gl) {
    const int64_t nb = b0 + ((j + 1) << level);
    const T* R = A.Rb + nb * kCB * kRW;
    const T* h = A.hp + nb * kCB;
#pragma unroll
    for (int t = 0; t < kCB; ++t) acc -= R[t * kRW + kCB + q] * h[t];
  }
  g[q] = acc;
}

template <typename T>
__global__ void cr_scatter_g_kernel(CRArgs<T> A, const double* g_in) {
  // padded g (xp) from a double vector over global columns; virtual columns 0
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A.total_blocks * kCB) return;
  const int64_t gb = e / kCB;
  const int q = (int)(e - gb * kCB);
  const int64_t k = inst_of_block(A.blk0, A.num_inst, gb);
  const int64_t col = kCB * (gb - A.blk0[k]) + q;
  A.xp[e] = col < A.cols[k] ? (T)g_in[A.col0[k] + col] : T(0);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side: instance tables, level work lists, launches.

struct CRPlan {
  int64_t num_inst = 0, total_blocks = 0;
  int splits = 1, levels = 0;
  bool thread_rows = true;   // compression by one thread per block (else one warp per split)
  std::vector<int64_t> lvl_off, lvl_n;     // eliminate / move / last items per level
  std::vector<int64_t> ev_off, ev_n;       // staying (even) blocks per level
  DevBuf tabs, items, evens, grp_lo, P, F0, F1, Rb, xp, hp;
  const int64_t* d_cols = nullptr;
  const int64_t* d_col0 = nullptr;
  const int64_t* d_row0 = nullptr;
  const int64_t* d_rows = nullptr;
  const int64_t* d_blk0 = nullptr;
};

void release_cr(CRPlan*& p) {
  if (!p) return;
  for (DevBuf* b : {&p->tabs, &p->items, &p->evens, &p->grp_lo, &p->P, &p->F0, &p->F1, &p->Rb, &p->xp, &p->hp})
    release(*b);
  delete p;
  p = nullptr;
}

qrkit_status cr_build(qrkit_ctx* ctx, CRPlan*& out, const std::vector<int64_t>& cols,
                      const std::vector<int64_t>& col0, const std::vector<int64_t>& row0,
                      const std::vector<int64_t>& rows) {
  release_cr(out);
  out = new CRPlan();
  CRPlan& C = *out;
  const int64_t ni = (int64_t)cols.size();
  C.num_inst = ni;
  std::vector<int64_t> blk0(ni + 1, 0);
  int64_t total_rows = 0;
  for (int64_t k = 0; k < ni; ++k) {
    if (cols[k] < 1) return fail(ctx, QRKIT_EINVAL, "banded instance without columns");
    blk0[k + 1] = blk0[k] + (cols[k] + kCB - 1) / kCB;
    total_rows += rows[k];
  }
  C.total_blocks = blk0[ni];
  if (C.total_blocks >= ((int64_t)1 << 30)) return fail(ctx, QRKIT_EUNSUPPORTED, "too many column blocks");
  const double per = C.total_blocks ? (double)total_rows / (double)C.total_blocks : 0.0;
  // few rows per column block: one thread per block merges its rows (little work per row);
  // row-heavy blocks: warps reduce 16 rows at a time, blocks split over several warps
  C.thread_rows = per <= 64.0;
  C.splits = C.thread_rows ? 1 : (int)std::min<double>(8.0, std::max<double>(1.0, std::ceil(per / 192.0)));
  // level work lists
  std::vector<std::vector<int64_t>> lv, ev;
  for (int64_t k = 0; k < ni; ++k) {
    const int64_t G = blk0[k + 1] - blk0[k];
    int64_t Gl = G;
    for (int l = 0;; ++l) {
      if ((int)lv.size() <= l) {
        lv.emplace_back();
        ev.emplace_back();
      }
      if (Gl == 1) {
        lv[l].push_back((k << 32) | (0 << 2) | 2);
        break;
      }
      for (int64_t i = 1; i < Gl; i += 2) lv[l].push_back((k << 32) | (i << 2) | 0);
      if (Gl % 2 == 1) lv[l].push_back((k << 32) | ((Gl - 1) << 2) | 1);
      for (int64_t j = 0; j < Gl; j += 2) ev[l].push_back((k << 32) | j);
      Gl = (Gl + 1) / 2;
    }
  }
  C.levels = (int)lv.size();
  std::vector<int64_t> items, evens;
  for (int l = 0; l < C.levels; ++l) {
    C.lvl_off.push_back((int64_t)items.size());
    C.lvl_n.push_back((int64_t)lv[l].size());
    items.insert(items.end(), lv[l].begin(), lv[l].end());
    C.ev_off.push_back((int64_t)evens.size());
    C.ev_n.push_back((int64_t)ev[l].size());
    evens.insert(evens.end(), ev[l].begin(), ev[l].end());
  }
  std::vector<int64_t> tabs;
  for (const auto* v : {&cols, &col0, &row0, &rows}) tabs.insert(tabs.end(), v->begin(), v->end());
  tabs.insert(tabs.end(), blk0.begin(), blk0.end());
  auto up = [&](DevBuf& d, const std::vector<int64_t>& h, const char* what) -> qrkit_status {
    qrkit_status r = ensure(ctx, d, std::max<size_t>(h.size(), 1) * sizeof(int64_t), what);
    if (r != QRKIT_OK) return r;
    if (!h.empty())
      QRKIT_CUDA_TRY(ctx, cudaMemcpy(d.ptr, h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    return QRKIT_OK;
  };
  qrkit_status rc;
  if ((rc = up(C.tabs, tabs, "banded tables")) != QRKIT_OK) return rc;
  if ((rc = up(C.items, items, "banded levels")) != QRKIT_OK) return rc;
  if ((rc = up(C.evens, evens, "banded levels")) != QRKIT_OK) return rc;
  const int64_t* t = (const int64_t*)C.tabs.ptr;
  C.d_cols = t;
  C.d_col0 = t + ni;
  C.d_row0 = t + 2 * ni;
  C.d_rows = t + 3 * ni;
  C.d_blk0 = t + 4 * ni;
  const size_t es = elem_size(ctx);
  const size_t TB = (size_t)C.total_blocks;
  if ((rc = ensure(ctx, C.grp_lo, TB * sizeof(int64_t), "banded group rows")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.P, TB * C.splits * 16 * kEW * es, "banded partial triangles")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.F0, TB * 16 * kEW * es, "banded block rows")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.F1, TB * 16 * kEW * es, "banded block rows")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.Rb, TB * kCB * kRW * es, "banded R blocks")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.xp, TB * kCB * es, "banded padded x")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.hp, TB * kCB * es, "banded padded h")) != QRKIT_OK) return rc;
  return QRKIT_OK;
}

qrkit_status cr_set_strategy(qrkit_ctx* ctx, CRPlan& C, bool thread_rows, int splits) {
  if (splits < 1 || splits > 64) return fail(ctx, QRKIT_EINVAL, "splits must be in [1, 64]");
  C.thread_rows = thread_rows;
  C.splits = thread_rows ? 1 : splits;
  return ensure(ctx, C.P, (size_t)C.total_blocks * C.splits * 16 * kEW * elem_size(ctx), "banded partial triangles");
}

template <typename T>
static CRArgs<T> cr_args(qrkit_ctx* ctx, CRPlan& C) {
  CRArgs<T> A{};
  A.num_inst = C.num_inst;
  A.cols = C.d_cols;
  A.col0 = C.d_col0;
  A.row0 = C.d_row0;
  A.rows = C.d_rows;
  A.blk0 = C.d_blk0;
  A.total_blocks = C.total_blocks;
  A.splits = C.splits;
  A.grp_lo = (int64_t*)C.grp_lo.ptr;
  A.P = (T*)C.P.ptr;
  A.F0 = (T*)C.F0.ptr;
  A.F1 = (T*)C.F1.ptr;
  A.Rb = (T*)C.Rb.ptr;
  A.xp = (T*)C.xp.ptr;
  A.hp = (T*)C.hp.ptr;
  A.status = ctx->d_status;
  return A;
}

#define CR_LAUNCH(ctx, ...)                         \
  do {                                              \
    __VA_ARGS__;                                    \
    (ctx)->launches += 1;                           \
    QRKIT_CUDA_TRY(ctx, cudaGetLastError());        \
  } while (0)

template <typename T>
static qrkit_status cr_solve_typed(qrkit_ctx* ctx, CRPlan& C, const int64_t* starts, int rpc, int w,
                                   const T* J, const T* b, const double* D, double lambda, T* x, double* res2) {
  cudaStream_t st = ctx->stream;
  CRArgs<T> A = cr_args<T>(ctx, C);
  A.starts = starts;
  A.rpc = rpc;
  A.w = w;
  A.J = J;
  A.b = b;
  A.D = D;
  A.lam = lambda;
  A.res2 = res2;
  QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(res2, 0, (size_t)C.num_inst * sizeof(double), st));
  if (starts) CR_LAUNCH(ctx, cr_ranges_kernel<T><<<nblk(C.total_blocks, 256), 256, 0, st>>>(A));
  const size_t tri_smem = (size_t)kTriElems * kCompThreads * sizeof(T);
  if (tri_smem > 48 * 1024) {
    QRKIT_CUDA_TRY(ctx, cudaFuncSetAttribute(cr_compress_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tri_smem));
  }
  if (C.thread_rows) {
    CR_LAUNCH(ctx, cr_compress_kernel<T><<<nblk(C.total_blocks, kCompThreads), kCompThreads, tri_smem, st>>>(A));
  } else {
    CR_LAUNCH(ctx, cr_compress_warp_kernel<T><<<nblk(C.total_blocks * C.splits * 32, 128), 128, 0, st>>>(A));
    CR_LAUNCH(ctx, cr_merge_warp_kernel<T><<<nblk(C.total_blocks * 32, 128), 128, 0, st>>>(A));
  }
  const int64_t* items = (const int64_t*)C.items.ptr;
  T* Fc = A.F0;
  T* Fn = A.F1;
  for (int l = 0; l < C.levels; ++l) {
    CR_LAUNCH(ctx, cr_level_kernel<T><<<nblk(C.lvl_n[l] * 32, 128), 128, 0, st>>>(A, items + C.lvl_off[l],
                                                                                 C.lvl_n[l], l, Fc, Fn));
    std::swap(Fc, Fn);
  }
  for (int l = C.levels - 1; l >= 0; --l)
    CR_LAUNCH(ctx, cr_backsub_kernel<T><<<nblk(C.lvl_n[l] * kItemThreads, 128), 128, 0, st>>>(
                       A, items + C.lvl_off[l], C.lvl_n[l], l, 0, x));
  return QRKIT_OK;
}

// dx = R^{-1} R^{-T} g with the stored factor (g: double over global columns).
template <typename T>
static qrkit_status cr_normal_typed(qrkit_ctx* ctx, CRPlan& C, const double* g, T* dx) {
  cudaStream_t st = ctx->stream;
  CRArgs<T> A = cr_args<T>(ctx, C);
  const int64_t* items = (const int64_t*)C.items.ptr;
  const int64_t* evens = (const int64_t*)C.evens.ptr;
  CR_LAUNCH(ctx, cr_scatter_g_kernel<T><<<nblk(C.total_blocks * kCB, 256), 256, 0, st>>>(A, g));
  for (int l = 0; l < C.levels; ++l) {
    CR_LAUNCH(ctx, cr_rt_kernel<T><<<nblk(C.lvl_n[l] * kItemThreads, 128), 128, 0, st>>>(A, items + C.lvl_off[l],
                                                                                          C.lvl_n[l], l));
    if (C.ev_n[l] > 0)
      CR_LAUNCH(ctx, cr_rt_update_kernel<T><<<nblk(C.ev_n[l] * kItemThreads, 128), 128, 0, st>>>(
                         A, evens + C.ev_off[l], C.ev_n[l], l));
  }
  for (int l = C.levels - 1; l >= 0; --l)
    CR_LAUNCH(ctx, cr_backsub_kernel<T><<<nblk(C.lvl_n[l] * kItemThreads, 128), 128, 0, st>>>(
                       A, items + C.lvl_off[l], C.lvl_n[l], l, 1, dx));
  return QRKIT_OK;
}

qrkit_status cr_solve(qrkit_ctx* ctx, CRPlan& C, const int64_t* starts, int rpc, int w, const void* J,
                      const void* b, const double* D, double lambda, void* x, double* res2) {
  if (w < 1 || w > kCB) return fail(ctx, QRKIT_EUNSUPPORTED, "the parallel banded QR needs w <= 8");
  if (ctx->precision == QRKIT_FP64)
    return cr_solve_typed<double>(ctx, C, starts, rpc, w, (const double*)J, (const double*)b, D, lambda,
                                  (double*)x, res2);
  return cr_solve_typed<float>(ctx, C, starts, rpc, w, (const float*)J, (const float*)b, D, lambda, (float*)x,
                               res2);
}

qrkit_status cr_normal_solve(qrkit_ctx* ctx, CRPlan& C, const double* g, void* dx) {
  if (ctx->precision == QRKIT_FP64) return cr_normal_typed<double>(ctx, C, g, (double*)dx);
  return cr_normal_typed<float>(ctx, C, g, (float*)dx);
}

}  // namespace qrkit
