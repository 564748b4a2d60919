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
  double* sums;          // or null: ||D p||^2, ||R'^{-T} D^2 p||^2, ||D^{-1} J^T b||^2 summed over blocks
};

// Stage 2 for one block: R (upper, m x m), c (m), d (m) -> p.  With sums, also the block's
// parts of the trust-region iteration (Moré 1977): ||D_i J_i^T b_i||-type term
// g2 = ||D_i^{-1} R_i^T c_i||^2 (= ||D_i^{-1} J_i^T b_i||^2, from stage 1's R and c),
// q2 = ||D_i p_i||^2 and z2 = ||z_i||^2 with R'_i^T z_i = D_i^2 p_i.
template <typename T>
__device__ __forceinline__ void more_block(T (&R)[kM][kM], T (&c)[kM], const T (&d)[kM], int m, double lambda,
                                           T* p, int* status, double* part) {
  if (part) {   // in the context precision (the bracket needs no more), squares summed in double
    double g2 = 0.0;
    for (int k = 0; k < m; ++k) {
      T gk = T(0);
      for (int i = 0; i <= k; ++i) gk += R[i][k] * c[i];
      gk /= d[k];
      g2 += (double)gk * (double)gk;
    }
    part[2] = g2;
  }
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
  if (part) {
    // q = D p; R'^T z = D q by forward substitution (R' upper triangular, now in R); z only
    // steers Newton's step, so it is formed in the context precision
    double q2 = 0.0, z2 = 0.0;
    T z[kM];
    for (int k = 0; k < m; ++k) {
      const T q = d[k] * c[k];
      q2 += (double)q * (double)q;
      T v = d[k] * q;
      for (int i = 0; i < k; ++i) v -= R[i][k] * z[i];
      z[k] = v / R[k][k];
      z2 += (double)z[k] * (double)z[k];
    }
    part[0] = q2;
    part[1] = z2;
  }
}

// The three sums of the trust-region iteration over a warp, then one atomic each.
__device__ __forceinline__ void more_sums_add(double* sums, double (&part)[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double v = part[j];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(sums + j, v);
  }
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
template <typename T, bool SUMS>
__global__ void __launch_bounds__(128) more_planes_kernel(MoreArgs<T> A) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = gid >> 5;
  const int slot = (int)(gid & 31);
  if (t >= A.num_tasks) return;   // warp-uniform: a warp is one task's slots
  const TaskHdr h = A.hdr[t];
  const int G = tasks::group_lanes(h.key), m = (h.key & 7) + 1;
  double part[3] = {0.0, 0.0, 0.0};
  if (slot < tasks::task_blocks(G)) {
    const TaskEntry e = A.ent[h.first + slot];
    if (e.n != 0) {
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
      more_block<T>(R, c, d, m, A.lambda, A.p + c0, A.status, SUMS ? part : nullptr);
    }
  }
  if constexpr (SUMS) more_sums_add(A.sums, part);
}

// Tile-mapping factor (J's packing): one thread per block.
template <typename T, bool SUMS>
__global__ void __launch_bounds__(128) more_packed_kernel(MoreArgs<T> A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double part[3] = {0.0, 0.0, 0.0};
  if (i < A.K) {
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
    more_block<T>(R, c, d, m, A.lambda, A.p + c0, A.status, SUMS ? part : nullptr);
  }
  if constexpr (SUMS) more_sums_add(A.sums, part);
}

template <typename T>
qrkit_status more_typed(qrkit_ctx* ctx, const void* qtb, const void* D, double lambda, void* p, double* sums) {
  const Plan& P = ctx->plan;
  MoreArgs<T> A{};
  A.qtb = (const T*)qtb;
  A.D = (const T*)D;
  A.lambda = lambda;
  A.p = (T*)p;
  A.status = ctx->d_status;
  A.sums = sums;
  if (ctx->factor_in_planes) {
    A.hdr = (const TaskHdr*)P.d_task_hdr.ptr;
    A.ent = (const TaskEntry*)P.d_task_ent.ptr;
    A.num_tasks = P.num_tasks;
    A.tF = (const T*)ctx->ws.tfactor.ptr;
    const int64_t threads = P.num_tasks * 32;
    if (sums)
      more_planes_kernel<T, true><<<(unsigned)((threads + 127) / 128), 128, 0, ctx->stream>>>(A);
    else
      more_planes_kernel<T, false><<<(unsigned)((threads + 127) / 128), 128, 0, ctx->stream>>>(A);
  } else {
    A.F = (const T*)ctx->ws.factor.ptr;
    A.val_off = (const int64_t*)P.d_val_off.ptr;
    A.row_off = (const int64_t*)P.d_row_off.ptr;
    A.col_off = (const int64_t*)P.d_col_off.ptr;
    A.n = (const uint8_t*)P.d_n.ptr;
    A.m = (const uint8_t*)P.d_m.ptr;
    A.K = P.K;
    if (sums)
      more_packed_kernel<T, true><<<(unsigned)((P.K + 127) / 128), 128, 0, ctx->stream>>>(A);
    else
      more_packed_kernel<T, false><<<(unsigned)((P.K + 127) / 128), 128, 0, ctx->stream>>>(A);
  }
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

}  // namespace

qrkit_status more_stage2(qrkit_ctx* ctx, const void* qtb, const void* D, double lambda, void* p) {
  if (ctx->precision == QRKIT_FP64) return more_typed<double>(ctx, qtb, D, lambda, p, nullptr);
  return more_typed<float>(ctx, qtb, D, lambda, p, nullptr);
}

// Moré's choice of lambda for a trust region of scaled radius delta (Moré 1977): stage 2 at
// lambda gives p, ||q|| = ||D p|| and ||z|| (R'^T z = D q), whose ratio fixes the derivative
// of the length, d||q||/dlambda = -||z||^2 / ||q||.  Newton's method on 1/||q|| - 1/delta,
// which is nearly linear in lambda: lambda += (||q|| / ||z||)^2 (||q|| - delta) / delta,
// kept inside a bracket [lo, hi] that each iterate narrows (lo from a Newton step of the
// convex, decreasing ||q|| - delta at 0, hi = ||D^{-1} J^T b|| / delta), until ||q|| is within
// sigma delta of delta; lambda = 0 when the Gauss-Newton step is already that short.  The three
// block sums come back to the host once per iteration (synchronous).
qrkit_status more_trust_region(qrkit_ctx* ctx, const void* qtb, const void* D, double delta, double sigma,
                               int max_iter, double* lambda, void* p, int* iterations) {
  DevBuf& S = ctx->more_sums;
  qrkit_status st = ensure(ctx, S, 3 * sizeof(double), "trust-region sums");
  if (st != QRKIT_OK) return st;
  double* sums = (double*)S.ptr;
  double h[3];
  auto eval = [&](double lam) -> qrkit_status {
    QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(sums, 0, 3 * sizeof(double), ctx->stream));
    qrkit_status r = ctx->precision == QRKIT_FP64 ? more_typed<double>(ctx, qtb, D, lam, p, sums)
                                                  : more_typed<float>(ctx, qtb, D, lam, p, sums);
    if (r != QRKIT_OK) return r;
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    QRKIT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return QRKIT_OK;
  };
  if ((st = eval(0.0)) != QRKIT_OK) return st;
  double qn = sqrt(h[0]), zn = sqrt(h[1]);
  const double gn = sqrt(h[2]);
  double phi = qn - delta;
  if (phi <= sigma * delta) {
    *lambda = 0.0;
    if (iterations) *iterations = 0;
    return QRKIT_OK;
  }
  double lo = zn > 0.0 ? phi * qn / (zn * zn) : 0.0;
  double hi = gn / delta;
  double lam = std::max(0.001 * hi, sqrt(lo * hi));
  for (int it = 1; it <= max_iter; ++it) {
    if ((st = eval(lam)) != QRKIT_OK) return st;
    qn = sqrt(h[0]);
    zn = sqrt(h[1]);
    phi = qn - delta;
    if (fabs(phi) <= sigma * delta || !(zn > 0.0)) {
      *lambda = lam;
      if (iterations) *iterations = it;
      return QRKIT_OK;
    }
    if (phi > 0.0) lo = std::max(lo, lam);
    else hi = std::min(hi, lam);
    const double next = lam + (qn / zn) * (qn / zn) * (phi / delta);
    lam = (lo < next && next < hi) ? next : std::max(0.001 * hi, sqrt(lo * hi));
  }
  *lambda = lam;
  if (iterations) *iterations = max_iter;
  return fail(ctx, QRKIT_ENOTCONV, "trust-region lambda: no convergence within max_iter iterations");
}

}  // namespace qrkit
