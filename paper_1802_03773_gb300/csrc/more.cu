// Moré's two-factorization Levenberg-Marquardt step (Sec. 5.2, Eq. LMTwoStep) for block-diagonal
// plans, stage 2: with J_i = Q_i R_i and c_i = the top m_i entries of Q_i^T b_i kept from the
// undamped fused solve (stage 1), each damping value costs only the QR of the 2 m_i x m_i stack
// [R_i; lambda^(1/2) D_i] with the damping row of column k interleaved after row k of R_i
// (Sec. 4.5), and R'_i p_i = top of Q'_i^T [c_i; 0].  Since ||J_i p - b_i||^2 = ||R_i p - c_i||^2
// + const, p_i is the minimiser of ||J_i p - b_i||^2 + lambda ||D_i p||^2 (Eq. 2).
//
// Mapping: one thread per block (m_i <= 8, the whole stack in registers).  The interleaved
// stack is reduced row by row: the damping row of column k has one non-zero, at column k, and
// is merged into rows k .. m-1 of the triangle by 2 x 2 reflections (each zeroes the row's
// leading entry against the diagonal of the triangle row, the row-merge form of a Householder
// reflection on a 2-vector), carrying the right-hand side.  The bottom entries of Q'^T [c; 0]
// so produced are the part of the residual that the damping adds.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "block_tasks.cuh"
#include "internal.h"

namespace qrkit {
namespace {

constexpr int kM = 8;

template <typename T>
struct MoreArgs {
  // the stored factor: task planes (warp-task mapping) or J's packing (tile mapping)
  const TaskHdr* hdr;
  const TaskEntry* ent;
  int64_t num_tasks;
  const T* tF;           // planes
  const T* F;            // J packing
  const int64_t* val_off;
  const int64_t* row_off;
  const int64_t* col_off;
  const uint8_t* n;
  const uint8_t* m;
  int64_t K;
  const T* qtb;          // J's row layout: c_i = qtb[row_off_i .. + m_i)
  const T* D;            // column layout or null (column norms of R_i = those of J_i)
  double lambda;
  T* p;
  int* status;
};

// Stage 2 for one block: R (upper, m x m), c (m), d (m) -> p.
template <typename T>
__device__ __forceinline__ void more_block(T (&R)[kM][kM], T (&c)[kM], const T (&d)[kM], int m, double lambda,
                                           T* p, int* status) {
  const T lh = (T)sqrt(lambda);
  for (int k = 0; k < m; ++k) {
    // the damping row of column k: one entry lambda^(1/2) d_k at column k, rhs 0
    T row[kM], rr = T(0);
#pragma unroll
    for (int j = 0; j < kM; ++j) row[j] = j == k ? lh * d[k] : T(0);
#pragma unroll
    for (int j = 0; j < kM; ++j) {
      if (j < k || j >= m) continue;
      const T a = R[j][j], bq = row[j];
      if (bq == T(0)) continue;
      // reflection on (a, bq): [a'; 0] with a' = -sign(a) sqrt(a^2 + bq^2)
      const T r = sqrt(a * a + bq * bq);
      const T beta = a >= T(0) ? -r : r;
      const T cs = a / beta, sn = bq / beta;   // H = [[cs, sn], [sn, -cs]]
      R[j][j] = beta;
      row[j] = T(0);
#pragma unroll
      for (int l = 0; l < kM; ++l) {
        if (l <= j || l >= m) continue;
        const T x = R[j][l], y = row[l];
        R[j][l] = cs * x + sn * y;
        row[l] = sn * x - cs * y;
      }
      const T x = c[j];
      c[j] = cs * x + sn * rr;
      rr = sn * x - cs * rr;
    }
  }
  bool ok = true;
  for (int k = m - 1; k >= 0; --k) {
    T s = c[k];
    for (int l = k + 1; l < m; ++l) s -= R[k][l] * c[l];
    if (R[k][k] == T(0)) ok = false;
    c[k] = s / R[k][k];
  }
  for (int k = 0; k < m; ++k) p[k] = c[k];
  if (!ok && status) atomicCAS(status, 0, (int)QRKIT_ESINGULAR);
}

template <typename T>
__device__ __forceinline__ void load_d(const MoreArgs<T>& A, const T (&R)[kM][kM], int64_t c0, int m, T (&d)[kM]) {
#pragma unroll
  for (int k = 0; k < kM; ++k) {
    if (k >= m) {
      d[k] = T(0);
    } else if (A.D) {
      d[k] = A.D[c0 + k];
    } else {   // column norm of J_i = column norm of R_i (Q_i orthogonal), zero -> 1
      T s = T(0);
      for (int i = 0; i <= k; ++i) s += R[i][k] * R[i][k];
      d[k] = s > T(0) ? sqrt(s) : T(1);
    }
  }
}

// Warp-task factor: one thread per task slot.
template <typename T>
__global__ void __launch_bounds__(128) more_planes_kernel(MoreArgs<T> A) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = gid >> 5;
  const int slot = (int)(gid & 31);
  if (t >= A.num_tasks) return;
  const TaskHdr h = A.hdr[t];
  const int G = tasks::group_lanes(h.key), m = (h.key & 7) + 1;
  if (slot >= tasks::task_blocks(G)) return;
  const TaskEntry e = A.ent[h.first + slot];
  if (e.n == 0) return;
  T R[kM][kM], c[kM], d[kM];
#pragma unroll
  for (int i = 0; i < kM; ++i)
#pragma unroll
    for (int j = 0; j < kM; ++j)
      R[i][j] = (i <= j && j < m) ? A.tF[((int64_t)h.plane + j) * kPlaneValues + slot * 4 * G + i] : T(0);
  const int64_t r0 = h.r0 + e.r, c0 = h.c0 + e.c;
#pragma unroll
  for (int k = 0; k < kM; ++k) c[k] = k < m ? A.qtb[r0 + k] : T(0);
  load_d<T>(A, R, c0, m, d);
  more_block<T>(R, c, d, m, A.lambda, A.p + c0, A.status);
}

// Tile-mapping factor (J's packing): one thread per block.
template <typename T>
__global__ void __launch_bounds__(128) more_packed_kernel(MoreArgs<T> A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.K) return;
  const int n = A.n[i], m = A.m[i];
  const T* F = A.F + A.val_off[i];
  T R[kM][kM], c[kM], d[kM];
#pragma unroll
  for (int r = 0; r < kM; ++r)
#pragma unroll
    for (int j = 0; j < kM; ++j) R[r][j] = (r <= j && j < m) ? F[(int64_t)j * n + r] : T(0);
  const int64_t r0 = A.row_off[i], c0 = A.col_off[i];
#pragma unroll
  for (int k = 0; k < kM; ++k) c[k] = k < m ? A.qtb[r0 + k] : T(0);
  load_d<T>(A, R, c0, m, d);
  more_block<T>(R, c, d, m, A.lambda, A.p + c0, A.status);
}

template <typename T>
qrkit_status more_typed(qrkit_ctx* ctx, const void* qtb, const void* D, double lambda, void* p) {
  const Plan& P = ctx->plan;
  MoreArgs<T> A{};
  A.qtb = (const T*)qtb;
  A.D = (const T*)D;
  A.lambda = lambda;
  A.p = (T*)p;
  A.status = ctx->d_status;
  if (ctx->factor_in_planes) {
    A.hdr = (const TaskHdr*)P.d_task_hdr.ptr;
    A.ent = (const TaskEntry*)P.d_task_ent.ptr;
    A.num_tasks = P.num_tasks;
    A.tF = (const T*)ctx->ws.tfactor.ptr;
    const int64_t threads = P.num_tasks * 32;
    more_planes_kernel<T><<<(unsigned)((threads + 127) / 128), 128, 0, ctx->stream>>>(A);
  } else {
    A.F = (const T*)ctx->ws.factor.ptr;
    A.val_off = (const int64_t*)P.d_val_off.ptr;
    A.row_off = (const int64_t*)P.d_row_off.ptr;
    A.col_off = (const int64_t*)P.d_col_off.ptr;
    A.n = (const uint8_t*)P.d_n.ptr;
    A.m = (const uint8_t*)P.d_m.ptr;
    A.K = P.K;
    more_packed_kernel<T><<<(unsigned)((P.K + 127) / 128), 128, 0, ctx->stream>>>(A);
  }
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

}  // namespace

qrkit_status more_stage2(qrkit_ctx* ctx, const void* qtb, const void* D, double lambda, void* p) {
  if (ctx->precision == QRKIT_FP64) return more_typed<double>(ctx, qtb, D, lambda, p);
  return more_typed<float>(ctx, qtb, D, lambda, p);
}

}  // namespace qrkit
